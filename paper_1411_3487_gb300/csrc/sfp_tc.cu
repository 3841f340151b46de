// sfp_tc.cu -- mode transforms of the SFP_FP32 path on the 5th-generation
// tensor cores (tcgen05), FP32-accurate through a three-pass TF32 split.
//
//   Out[j][i] = sum_k In[j][k] * B[i][k]        (NT: both operands K-contiguous)
//   inverse (Eq. e5):  In = R   [3C][M], B = chi   [n][p]  -> Out = u (bonds)
//   forward (Eq. c4):  In = f|z [6C][M], B = phi^T [p][n]  -> Out = DeltaH|Z
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
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
          const __grid_constant__ CUtensorMap tmBl, float* __restrict__ Out, int J, int M, int* err)
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
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmBh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmBl)) : "memory");
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
                tma_load_2d(st, &tmA, &full[s], kb * kKB, row0);
                tma_load_2d(st + 2 * S::kA, &tmBh, &full[s], kb * kKB, col0);
                tma_load_2d(st + 2 * S::kA + S::kB, &tmBl, &full[s], kb * kKB, col0);
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
                    float4* o = (float4*)(Out + (size_t)row * M + col0 + c);
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

}  // namespace

struct TcPlan {
    int M = 0, rows = 0, NT = 0;
    float* B[4] = {nullptr, nullptr, nullptr, nullptr};   // chi_hi, chi_lo, phiT_hi, phiT_lo
    CUtensorMap mapA[2], mapBh[2], mapBl[2];
    float* out[2] = {nullptr, nullptr};
    int* err = nullptr;
};

bool tc_supported(int M) { return M == 32 || M == 64 || M == 128 || M == 256 || M == 512; }

int tc_create(TcPlan** out, int M, int rows, const double* phi, const double* phiT, const float* R,
              float* r_out, const float* fz, float* yz_out, int* err, cudaStream_t stream)
{
    *out = nullptr;
    if (!tc_supported(M)) return report(SFP_ENOTSUP, "tensor-core transforms need M in {32, 64, 128, 256, 512}");
    TcPlan* p = new TcPlan();
    p->M = M;
    p->rows = rows;
    p->NT = M <= 256 ? M : 256;
    p->err = err;
    const size_t n = (size_t)M * M;
    std::vector<float> hi(n), lo(n);
    for (int t = 0; t < 2; ++t) {
        const double* src = t == 0 ? phi : phiT;
        for (size_t i = 0; i < n; ++i) {
            hi[i] = ptx::tf32_round_host(src[i]);
            lo[i] = ptx::tf32_round_host(src[i] - (double)hi[i]);
        }
        for (int k = 0; k < 2; ++k) {
            if (cudaMalloc(&p->B[2 * t + k], n * sizeof(float)) != cudaSuccess) {
                tc_destroy(p);
                return report(SFP_ENOMEM, "tensor-core table allocation failed");
            }
            if (cudaMemcpyAsync(p->B[2 * t + k], k == 0 ? hi.data() : lo.data(), n * sizeof(float),
                                cudaMemcpyHostToDevice, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                tc_destroy(p);
                return report(SFP_ECUDA, "tensor-core table upload failed");
            }
        }
    }
    int rc;
    // inverse: A = R [rows][M], B = chi ; forward: A = f|z [2 rows][M], B = phi^T
    if ((rc = make_map(&p->mapA[0], R, rows, M, kRows)) || (rc = make_map(&p->mapA[1], fz, 2 * rows, M, kRows)) ||
        (rc = make_map(&p->mapBh[0], p->B[0], M, M, p->NT)) || (rc = make_map(&p->mapBl[0], p->B[1], M, M, p->NT)) ||
        (rc = make_map(&p->mapBh[1], p->B[2], M, M, p->NT)) || (rc = make_map(&p->mapBl[1], p->B[3], M, M, p->NT))) {
        tc_destroy(p);
        return rc;
    }
    p->out[0] = r_out;
    p->out[1] = yz_out;
    cudaError_t e = cudaSuccess;
    switch (p->NT) {
        case 32: e = cudaFuncSetAttribute(k_tc_gemm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<32>::kBytes); break;
        case 64: e = cudaFuncSetAttribute(k_tc_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<64>::kBytes); break;
        case 128: e = cudaFuncSetAttribute(k_tc_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<128>::kBytes); break;
        case 256: e = cudaFuncSetAttribute(k_tc_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<256>::kBytes); break;
        default: e = cudaErrorInvalidValue; break;
    }
    if (e != cudaSuccess) {
        tc_destroy(p);
        return report(SFP_ECUDA, "cudaFuncSetAttribute failed");
    }
    *out = p;
    return SFP_OK;
}

int tc_transform(TcPlan* p, int which, cudaStream_t stream)
{
    const int J = which == 0 ? p->rows : 2 * p->rows;
    dim3 grid((J + kRows - 1) / kRows, p->M / p->NT);
    switch (p->NT) {
        case 32:
            k_tc_gemm<32><<<grid, kThreads, Smem<32>::kBytes, stream>>>(p->mapA[which], p->mapBh[which], p->mapBl[which], p->out[which], J, p->M, p->err);
            break;
        case 64:
            k_tc_gemm<64><<<grid, kThreads, Smem<64>::kBytes, stream>>>(p->mapA[which], p->mapBh[which], p->mapBl[which], p->out[which], J, p->M, p->err);
            break;
        case 128:
            k_tc_gemm<128><<<grid, kThreads, Smem<128>::kBytes, stream>>>(p->mapA[which], p->mapBh[which], p->mapBl[which], p->out[which], J, p->M, p->err);
            break;
        case 256:
            k_tc_gemm<256><<<grid, kThreads, Smem<256>::kBytes, stream>>>(p->mapA[which], p->mapBh[which], p->mapBl[which], p->out[which], J, p->M, p->err);
            break;
        default:
            return report(SFP_ENOTSUP, "unsupported tile width");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report(SFP_ECUDA, cudaGetErrorString(e));
    return SFP_OK;
}

size_t tc_bytes(const TcPlan* p) { return p ? (size_t)4 * p->M * p->M * sizeof(float) : 0; }

void tc_destroy(TcPlan* p)
{
    if (!p) return;
    for (float* b : p->B)
        if (b) cudaFree(b);
    delete p;
}

}  // namespace sfp
