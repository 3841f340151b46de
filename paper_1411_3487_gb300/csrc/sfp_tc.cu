// sfp_tc.cu -- mode transforms of the SFP_FP32 path on the 5th-generation
// tensor cores (tcgen05), FP32-accurate through a three-pass TF32 split.
//
//   Out[j][i] = sum_k In[j][k] * B[i][k]        (NT: both operands K-contiguous)
//   inverse (Eq. e5):       In = R [3C][M], B = chi   [n][p]  -> Out = u (bonds)
//   forward (Eqs. e11, c4): In = v [3C][M], B = chi^T [p][n]  -> Out = DeltaH
//                           In = z [3C][M], B = phi^T [p][n]  -> Out = Z
// The two halves of the forward transform are one launch: blockIdx.z picks
// the half (its rows of In and Out, and its table).
//
// Each CTA owns 128 rows j (one UMMA M = 128 tile) and NT output columns
// (NT = M up to 256; M = 512 uses two column tiles).  The K loop runs over
// 32-wide blocks (one 128-byte swizzle atom of FP32):
//   warp 0      TMA producer: In tile (FP32) and B_hi / B_lo tiles -> smem
//   warps 2..5  split the In tile in place into hi = rna_tf32(x) and lo = x - hi
//   warp 1      one thread issues D += A_hi B_lo + A_lo B_hi + A_hi B_hi
//               (tcgen05.mma kind::tf32, FP32 accumulator in TMEM)
//   warps 2..5  epilogue: tcgen05.ld rows of D -> FP32 global stores
// The dropped A_lo B_lo term is below 2^-21 relative.  B_hi / B_lo are split
// once on the host from the FP64 tables.  Every mbarrier wait is bounded; on
// timeout the CTA raises bit 2 of the error word, skips its remaining work,
// frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/sfp.h"
#include "sfp_tc.h"
#include "sfp_ptx.cuh"

namespace sfp {
namespace {

using namespace ptx;

constexpr int kRows = 128;          // UMMA M
constexpr int kKB = 32;             // K block: 32 FP32 = one 128-byte swizzle row
constexpr int kStages = 2;
constexpr int kThreads = 192;       // 6 warps

template <int NT>
struct Smem {
    static constexpr int kA = kRows * kKB * 4;       // 16 KB
    static constexpr int kB = NT * kKB * 4;          // NT * 128 B
    static constexpr int kStage = 2 * kA + 2 * kB;   // A hi, A lo, B hi, B lo
    static constexpr int kBytes = kStages * kStage + 1024 /* barriers */ + 1024 /* alignment slack */;
};

template <int NT>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh0,
          const __grid_constant__ CUtensorMap tmBl0, const __grid_constant__ CUtensorMap tmBh1,
          const __grid_constant__ CUtensorMap tmBl1, float* __restrict__ Out, int J, int M, int* err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    using S = Smem<NT>;
    uint64_t* bars = (uint64_t*)(smem + kStages * S::kStage);
    uint64_t* full = bars;                  // TMA landed          (count 1 + tx)
    uint64_t* conv = bars + kStages;        // A split into hi/lo  (count 128)
    uint64_t* empty = bars + 2 * kStages;   // MMAs done with stage (commit)
    uint64_t* done = bars + 3 * kStages;    // all MMAs done        (commit)
    uint32_t* tmem_slot = (uint32_t*)(bars + 3 * kStages + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * kRows;
    const int col0 = blockIdx.y * NT;
    const int roff = blockIdx.z * J;    // first row of this half in In and Out
    const CUtensorMap* tmBh = blockIdx.z ? &tmBh1 : &tmBh0;
    const CUtensorMap* tmBl = blockIdx.z ? &tmBl1 : &tmBl0;
    const int nk = (M + kKB - 1) / kKB;
    constexpr uint32_t kCols = NT < 32 ? 32 : NT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 128);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmBh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmBl)) : "memory");
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

    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages;
                const uint32_t ph = (kb / kStages) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1, err, abort_flag)) break;
                uint8_t* st = smem + s * S::kStage;
                mbar_expect_tx(&full[s], S::kA + 2 * S::kB);
                tma_load_2d(st, &tmA, &full[s], kb * kKB, roff + row0);
                tma_load_2d(st + 2 * S::kA, tmBh, &full[s], kb * kKB, col0);
                tma_load_2d(st + 2 * S::kA + S::kB, tmBl, &full[s], kb * kKB, col0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(kRows, NT);
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages;
                const uint32_t ph = (kb / kStages) & 1;
                if (!mbar_wait(&conv[s], ph, err, abort_flag)) break;
                fence_after();
                const uint32_t st = smem_u32(smem + s * S::kStage);
                const uint32_t a_hi = st, a_lo = st + S::kA, b_hi = st + 2 * S::kA, b_lo = b_hi + S::kB;
#pragma unroll
                for (int kk = 0; kk < kKB / 8; ++kk) {
                    const uint32_t off = kk * 32;   // 8 TF32 = 32 bytes along K
                    mma_tf32(tmem, sdesc(a_hi + off), sdesc(b_lo + off), idesc, (kb | kk) != 0);
                    mma_tf32(tmem, sdesc(a_lo + off), sdesc(b_hi + off), idesc, 1);
                    mma_tf32(tmem, sdesc(a_hi + off), sdesc(b_hi + off), idesc, 1);
                }
                mma_commit(&empty[s]);
            }
            mma_commit(done);
        }
    } else {
        // warps 2..5: split the A tile of each stage, then the epilogue
        const int t = threadIdx.x - 64;   // 0..127
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            const uint32_t ph = (kb / kStages) & 1;
            if (!mbar_wait(&full[s], ph, err, abort_flag)) break;
            float4* a = (float4*)(smem + s * S::kStage);
            float4* al = (float4*)(smem + s * S::kStage + S::kA);
#pragma unroll
            for (int i = 0; i < S::kA / 16 / 128; ++i) {
                const int e = t + 128 * i;
                const float4 x = a[e];
                float4 h, l;
                h.x = tf32_rna(x.x); l.x = tf32_rna(x.x - h.x);
                h.y = tf32_rna(x.y); l.y = tf32_rna(x.y - h.y);
                h.z = tf32_rna(x.z); l.z = tf32_rna(x.z - h.z);
                h.w = tf32_rna(x.w); l.w = tf32_rna(x.w - h.w);
                a[e] = h;
                al[e] = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv[s]);
        }
        // epilogue: lane quarter q = warp % 4 holds rows 32q .. 32q+31 of D
        const bool ok = mbar_wait(done, 0, err, abort_flag);
        fence_after();
        const int q = warp & 3;
        const int row = row0 + 32 * q + lane;
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < NT; c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
                if (row < J) {
                    float4* o = (float4*)(Out + (size_t)(roff + row) * M + col0 + c);
                    o[0] = make_float4(v[0], v[1], v[2], v[3]);
                    o[1] = make_float4(v[4], v[5], v[6], v[7]);
                    o[2] = make_float4(v[8], v[9], v[10], v[11]);
                    o[3] = make_float4(v[12], v[13], v[14], v[15]);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

int make_map(CUtensorMap* m, const float* base, int rows, int cols, int box_rows)
{
    return make_map_2d(m, base, rows, cols, box_rows);
}

// ---------------------------------------------------------------------------
// BF16 variant (SFP_MIXED_BF16): the FP32 A tile (TMA, 128-byte swizzle) is
// split by threads into BF16 hi = rn(x) and lo = rn(x - hi) in 64-byte-swizzled
// K-major tiles; the tables are BF16 hi/lo from the host; three kind::f16 passes
// per K step (A_hi B_lo + A_lo B_hi + A_hi B_hi), FP32 accumulate.  About 16 bits
// per product instead of the TF32 split's 21.
// ---------------------------------------------------------------------------
constexpr int kStagesBf = 3;

template <int NT>
struct SmemBf {
    static constexpr int kA32 = kRows * kKB * 4;     // FP32 tile from TMA, 16 KB
    static constexpr int kA = kRows * kKB * 2;       // BF16 tile, 8 KB
    static constexpr int kB = NT * kKB * 2;          // BF16 table tile, NT x 64 B
    static constexpr int kStage = kA32 + 2 * kA + 2 * kB;
    static constexpr int kBytes = kStagesBf * kStage + 1024 + 1024;
};

__device__ __forceinline__ uint32_t swz128(int r, int k) { return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) << 4)) + ((k & 3) << 2)); }

__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

template <int NT, bool TWO = false>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh0,
          const __grid_constant__ CUtensorMap tmBl0, const __grid_constant__ CUtensorMap tmBh1,
          const __grid_constant__ CUtensorMap tmBl1, float* __restrict__ Out, int J, int M, int* err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    using S = SmemBf<NT>;
    constexpr int ST = kStagesBf;
    uint64_t* bars = (uint64_t*)(smem + ST * S::kStage);
    uint64_t* full = bars;
    uint64_t* conv = bars + ST;
    uint64_t* empty = bars + 2 * ST;
    uint64_t* done = bars + 3 * ST;
    uint32_t* tmem_slot = (uint32_t*)(bars + 3 * ST + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * kRows;
    const int col0 = blockIdx.y * NT;
    const int roff = blockIdx.z * J;    // first row of this half in In and Out
    const CUtensorMap* tmBh = blockIdx.z ? &tmBh1 : &tmBh0;
    const CUtensorMap* tmBl = blockIdx.z ? &tmBl1 : &tmBl0;
    const int nk = (M + kKB - 1) / kKB;
    constexpr uint32_t kCols = NT < 32 ? 32 : NT;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 128);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmBh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmBl)) : "memory");
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

    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % ST;
                const uint32_t ph = (kb / ST) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1, err, abort_flag)) break;
                uint8_t* st = smem + s * S::kStage;
                uint8_t* bh = st + S::kA32 + 2 * S::kA;
                mbar_expect_tx(&full[s], S::kA32 + 2 * S::kB);
                tma_load_2d(st, &tmA, &full[s], kb * kKB, roff + row0);
                tma_load_2d(bh, tmBh, &full[s], kb * kKB, col0);
                tma_load_2d(bh + S::kB, tmBl, &full[s], kb * kKB, col0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::f16, BF16 A and B, FP32 accumulate, both K-major
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                       ((uint32_t)(kRows >> 4) << 24);
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % ST;
                const uint32_t ph = (kb / ST) & 1;
                if (!mbar_wait(&conv[s], ph, err, abort_flag)) break;
                fence_after();
                const uint32_t st = smem_u32(smem + s * S::kStage);
                const uint32_t a_hi = st + S::kA32, a_lo = a_hi + S::kA, b_hi = a_lo + S::kA, b_lo = b_hi + S::kB;
#pragma unroll
                for (int kk = 0; kk < kKB / 16; ++kk) {
                    const uint32_t off = kk * 32;   // 16 BF16 = 32 bytes along K
                    const uint32_t acc = (kb | kk) != 0;
                    if constexpr (!TWO)   // TWO: the tables as their BF16 hi part alone
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                     ::"r"(tmem), "l"(sdesc64(a_hi + off)), "l"(sdesc64(b_lo + off)), "r"(idesc), "r"(acc) : "memory");
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                 ::"r"(tmem), "l"(sdesc64(a_lo + off)), "l"(sdesc64(b_hi + off)), "r"(idesc), "r"(TWO ? acc : 1u) : "memory");
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                 ::"r"(tmem), "l"(sdesc64(a_hi + off)), "l"(sdesc64(b_hi + off)), "r"(idesc), "r"(1u) : "memory");
                }
                mma_commit(&empty[s]);
            }
            mma_commit(done);
        }
    } else {
        // warps 2..5: thread t converts row t of each FP32 tile into BF16 hi / lo
        const int t = threadIdx.x - 64;   // 0..127
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % ST;
            const uint32_t ph = (kb / ST) & 1;
            if (!mbar_wait(&full[s], ph, err, abort_flag)) break;
            const uint8_t* a32 = smem + s * S::kStage;
            uint8_t* ah = smem + s * S::kStage + S::kA32;
            uint8_t* al = ah + S::kA;
#pragma unroll
            for (int c = 0; c < 4; ++c) {          // 16-byte chunks of 8 BF16
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float4 x = *reinterpret_cast<const float4*>(a32 + swz128(t, 8 * c + 4 * q));
                    const float xs[4] = {x.x, x.y, x.z, x.w};
                    uint16_t h[4], l[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        h[i] = bf16_bits(xs[i]);
                        l[i] = bf16_bits(xs[i] - __bfloat162float(__ushort_as_bfloat16(h[i])));
                    }
                    hw[2 * q] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
                    hw[2 * q + 1] = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
                    lw[2 * q] = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
                    lw[2 * q + 1] = (uint32_t)l[2] | ((uint32_t)l[3] << 16);
                }
                const uint32_t o = (uint32_t)(t * 64 + ((c ^ ((t >> 1) & 3)) << 4));
                *reinterpret_cast<uint4*>(ah + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(al + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&conv[s]);
        }
        const bool ok = mbar_wait(done, 0, err, abort_flag);
        fence_after();
        const int q = warp & 3;
        const int row = row0 + 32 * q + lane;
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < NT; c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
                if (row < J) {
                    float4* o = (float4*)(Out + (size_t)(roff + row) * M + col0 + c);
                    o[0] = make_float4(v[0], v[1], v[2], v[3]);
                    o[1] = make_float4(v[4], v[5], v[6], v[7]);
                    o[2] = make_float4(v[8], v[9], v[10], v[11]);
                    o[3] = make_float4(v[12], v[13], v[14], v[15]);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

}  // namespace

struct TcPlan {
    int M = 0, rows = 0, NT = 0;
    bool bf16 = false, two = false;
    // tables t = 0: chi (inverse), 1: chi^T (forward, force half), 2: phi^T
    // (forward, noise half); B[2 t] hi, B[2 t + 1] lo (FP32 or BF16)
    void* B[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    CUtensorMap mapA[2], mapBh[3], mapBl[3];
    float* out[2] = {nullptr, nullptr};
    int* err = nullptr;
};

bool tc_supported(int M) { return M == 32 || M == 64 || M == 128 || M == 256 || M == 512; }

int tc_create(TcPlan** out, int M, int rows, const double* chi, const double* chiT, const double* phiT,
              const float* R, float* r_out, const float* fz, float* yz_out, int* err, cudaStream_t stream, bool bf16,
              bool two)
{
    *out = nullptr;
    if (!tc_supported(M)) return report(SFP_ENOTSUP, "tensor-core transforms need M in {32, 64, 128, 256, 512}");
    TcPlan* p = new TcPlan();
    p->M = M;
    p->rows = rows;
    p->NT = M <= 256 ? M : 256;
    p->err = err;
    p->bf16 = bf16;
    p->two = bf16 && two;
    const size_t n = (size_t)M * M;
    const double* src[3] = {chi, chiT, phiT};
    const size_t el = bf16 ? 2 : sizeof(float);
    for (int t = 0; t < 3; ++t) {
        std::vector<float> hi(bf16 ? 0 : n), lo(bf16 ? 0 : n);
        std::vector<uint16_t> hb(bf16 ? n : 0), lb(bf16 ? n : 0);
        for (size_t i = 0; i < n; ++i) {
            if (bf16) {
                hb[i] = bf16_round_host((float)src[t][i]);
                lb[i] = bf16_round_host((float)(src[t][i] - (double)bf16_to_float_host(hb[i])));
            } else {
                hi[i] = ptx::tf32_round_host(src[t][i]);
                lo[i] = ptx::tf32_round_host(src[t][i] - (double)hi[i]);
            }
        }
        for (int k = 0; k < 2; ++k) {
            const void* h = bf16 ? (const void*)(k == 0 ? hb.data() : lb.data())
                                 : (const void*)(k == 0 ? hi.data() : lo.data());
            if (cudaMalloc(&p->B[2 * t + k], n * el) != cudaSuccess) {
                tc_destroy(p);
                return report(SFP_ENOMEM, "tensor-core table allocation failed");
            }
            if (cudaMemcpyAsync(p->B[2 * t + k], h, n * el, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                tc_destroy(p);
                return report(SFP_ECUDA, "tensor-core table upload failed");
            }
        }
    }
    // inverse: A = R [rows][M]; forward: A = v | z [2 rows][M] (a half per blockIdx.z)
    int rc = make_map(&p->mapA[0], R, rows, M, kRows);
    if (!rc) rc = make_map(&p->mapA[1], fz, 2 * rows, M, kRows);
    for (int t = 0; t < 3 && !rc; ++t) {
        if (bf16) {
            rc = make_map_bf16(&p->mapBh[t], p->B[2 * t], M, M, p->NT);
            if (!rc) rc = make_map_bf16(&p->mapBl[t], p->B[2 * t + 1], M, M, p->NT);
        } else {
            rc = make_map(&p->mapBh[t], (const float*)p->B[2 * t], M, M, p->NT);
            if (!rc) rc = make_map(&p->mapBl[t], (const float*)p->B[2 * t + 1], M, M, p->NT);
        }
    }
    if (rc) {
        tc_destroy(p);
        return rc;
    }
    p->out[0] = r_out;
    p->out[1] = yz_out;
    cudaError_t e = cudaSuccess;
#define SFP_TC_ATTR(K, S) cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes)
    switch (p->NT + (bf16 ? 1 : 0)) {
        case 32: e = SFP_TC_ATTR(k_tc_gemm<32>, Smem<32>); break;
        case 64: e = SFP_TC_ATTR(k_tc_gemm<64>, Smem<64>); break;
        case 128: e = SFP_TC_ATTR(k_tc_gemm<128>, Smem<128>); break;
        case 256: e = SFP_TC_ATTR(k_tc_gemm<256>, Smem<256>); break;
        case 33: e = p->two ? SFP_TC_ATTR((k_tc_gemm_bf16<32, true>), SmemBf<32>) : SFP_TC_ATTR(k_tc_gemm_bf16<32>, SmemBf<32>); break;
        case 65: e = p->two ? SFP_TC_ATTR((k_tc_gemm_bf16<64, true>), SmemBf<64>) : SFP_TC_ATTR(k_tc_gemm_bf16<64>, SmemBf<64>); break;
        case 129: e = p->two ? SFP_TC_ATTR((k_tc_gemm_bf16<128, true>), SmemBf<128>) : SFP_TC_ATTR(k_tc_gemm_bf16<128>, SmemBf<128>); break;
        case 257: e = p->two ? SFP_TC_ATTR((k_tc_gemm_bf16<256, true>), SmemBf<256>) : SFP_TC_ATTR(k_tc_gemm_bf16<256>, SmemBf<256>); break;
        default: e = cudaErrorInvalidValue; break;
    }
#undef SFP_TC_ATTR
    if (e != cudaSuccess) {
        tc_destroy(p);
        return report(SFP_ECUDA, "cudaFuncSetAttribute failed");
    }
    *out = p;
    return SFP_OK;
}

int tc_transform(TcPlan* p, int which, cudaStream_t stream)
{
    // inverse: one table over the rows of R; forward: the force half (chi^T) and
    // the noise half (phi^T) of [v | z] as grid z = 0, 1; which = 2: the force
    // half alone (mode-keyed noise, whose Z needs no projection)
    if (which < 0 || which > 2) return report(SFP_EINVAL, "tc_transform: which must be 0, 1 or 2");
    const int J = p->rows;
    const dim3 grid((J + kRows - 1) / kRows, p->M / p->NT, which == 1 ? 2 : 1);
    const int b0 = which == 0 ? 0 : 1, b1 = which == 0 ? 0 : which == 1 ? 2 : 1;
    which = which == 0 ? 0 : 1;
#define SFP_TC_LAUNCH(K, S)                                                                             \
    K<<<grid, kThreads, S::kBytes, stream>>>(p->mapA[which], p->mapBh[b0], p->mapBl[b0], p->mapBh[b1], \
                                            p->mapBl[b1], p->out[which], J, p->M, p->err)
#define SFP_TC_LAUNCH_BF(NTV)                                                                           \
    if (p->two)                                                                                          \
        k_tc_gemm_bf16<NTV, true><<<grid, kThreads, SmemBf<NTV>::kBytes, stream>>>(                     \
            p->mapA[which], p->mapBh[b0], p->mapBl[b0], p->mapBh[b1], p->mapBl[b1], p->out[which], J, p->M, p->err); \
    else                                                                                                 \
        k_tc_gemm_bf16<NTV><<<grid, kThreads, SmemBf<NTV>::kBytes, stream>>>(                           \
            p->mapA[which], p->mapBh[b0], p->mapBl[b0], p->mapBh[b1], p->mapBl[b1], p->out[which], J, p->M, p->err)
    switch (p->NT + (p->bf16 ? 1 : 0)) {
        case 32: SFP_TC_LAUNCH(k_tc_gemm<32>, Smem<32>); break;
        case 64: SFP_TC_LAUNCH(k_tc_gemm<64>, Smem<64>); break;
        case 128: SFP_TC_LAUNCH(k_tc_gemm<128>, Smem<128>); break;
        case 256: SFP_TC_LAUNCH(k_tc_gemm<256>, Smem<256>); break;
        case 33: SFP_TC_LAUNCH_BF(32); break;
        case 65: SFP_TC_LAUNCH_BF(64); break;
        case 129: SFP_TC_LAUNCH_BF(128); break;
        case 257: SFP_TC_LAUNCH_BF(256); break;
        default: return report(SFP_ENOTSUP, "unsupported tile width");
    }
#undef SFP_TC_LAUNCH
#undef SFP_TC_LAUNCH_BF
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report(SFP_ECUDA, cudaGetErrorString(e));
    return SFP_OK;
}

size_t tc_bytes(const TcPlan* p) { return p ? (size_t)6 * p->M * p->M * (p->bf16 ? 2 : sizeof(float)) : 0; }

void tc_destroy(TcPlan* p)
{
    if (!p) return;
    for (void* b : p->B)
        if (b) cudaFree(b);
    delete p;
}

}  // namespace sfp
