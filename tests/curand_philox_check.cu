// curand_philox_check.cu -- test helper: raw Philox4x32-10 words from cuRAND's
// device API, as a third implementation of the generator beside the CUDA
// library's and the oracle's.  Built by tests/test_philox_curand_gpu.py.
//
// cuRAND's Philox state takes a 64-bit seed as its key (low word first) and
// counts with a 128-bit counter whose high 64 bits are the subsequence and
// whose low 64 bits advance by one per four outputs (offset / 4).  So the
// words for counter (step_lo, step_hi, i, tag) and key (seed, job) are the
// first four outputs after curand_init(seed | job << 32, i | tag << 32,
// 4 * step).
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_curand_words(uint32_t seed, uint32_t job, unsigned long long step, uint32_t tag, int n,
                               uint4* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init((unsigned long long)seed | ((unsigned long long)job << 32),
                (unsigned long long)(uint32_t)i | ((unsigned long long)tag << 32), 4ull * step, &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_words(uint32_t seed, uint32_t job, unsigned long long step, uint32_t tag, int count,
                                   uint32_t* host_out)
{
    uint4* d = nullptr;
    if (count <= 0 || cudaMalloc(&d, (size_t)count * sizeof(uint4)) != cudaSuccess) return -1;
    k_curand_words<<<(count + 127) / 128, 128>>>(seed, job, step, tag, count, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, (size_t)count * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : -1;
}
