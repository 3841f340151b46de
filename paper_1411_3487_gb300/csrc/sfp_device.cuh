// sfp_device.cuh -- device helpers shared by the kernels of the GB300 path:
// the counter-based noise generator and the per-bead normals.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sfp {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies with a Weyl-sequence key schedule.  Counter
// (step_lo, step_hi, index, tag), key (seed, job_id).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        // each multiply as one 32 x 32 -> 64-bit product (both halves at once)
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Open-interval uniform from the top 23 bits: exact in FP32 and FP64, so the
// FP32 and FP64 paths see bit-identical uniforms.
__device__ __forceinline__ float u01f(uint32_t x)
{
    return (float)(x >> 9) * 1.1920928955078125e-07f + 5.9604644775390625e-08f;
}
__device__ __forceinline__ double u01d(uint32_t x)
{
    return (double)(x >> 9) * 1.1920928955078125e-07 + 5.9604644775390625e-08;
}

// Bead noise (Eq. b5).  The normals of one chain and step are numbered
// k = 3 n + alpha (bead n, axis alpha); normal k is value k % 4 of Philox call
// k / 4, counter (step_lo, step_hi, call, tag), key (seed, job).  A call gives
// four normals by Box-Muller on its word pairs (0,1) and (2,3), both values of
// each pair used.  Beads 4t .. 4t+3 (12 normals) take exactly calls 3t .. 3t+2.
template <typename T> struct Normals;
template <> struct Normals<float> {
    static __device__ __forceinline__ void draw4(uint32_t seed, uint32_t job, int64_t step,
                                                 uint32_t call, uint32_t tag, float g[4])
    {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), call, tag), make_uint2(seed, job));
        // sqrt(t) as t rsqrt(t) (t >= 2^-23 here, never zero or denormal)
        const float ta = -2.0f * logf(u01f(w.x)), tb = -2.0f * logf(u01f(w.z));
        const float ra = ta * rsqrtf(ta), rb = tb * rsqrtf(tb);
        float sa, ca, sb, cb;
        sincospif(2.0f * u01f(w.y), &sa, &ca);
        sincospif(2.0f * u01f(w.w), &sb, &cb);
        g[0] = ra * ca; g[1] = ra * sa; g[2] = rb * cb; g[3] = rb * sb;
    }
};
template <> struct Normals<double> {
    static __device__ __forceinline__ void draw4(uint32_t seed, uint32_t job, int64_t step,
                                                 uint32_t call, uint32_t tag, double g[4])
    {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), call, tag), make_uint2(seed, job));
        const double ra = sqrt(-2.0 * log(u01d(w.x)));
        const double rb = sqrt(-2.0 * log(u01d(w.z)));
        double sa, ca, sb, cb;
        sincospi(2.0 * u01d(w.y), &sa, &ca);
        sincospi(2.0 * u01d(w.w), &sb, &cb);
        g[0] = ra * ca; g[1] = ra * sa; g[2] = rb * cb; g[3] = rb * sb;
    }
};

// The normals of beads 4t .. 4t+3 of one chain and step: z[alpha][i] is bead
// 4t + i, axis alpha (calls 3t, 3t+1, 3t+2).
template <typename T>
__device__ __forceinline__ void bead_quad_normals(uint32_t seed, uint32_t job, int64_t step, uint32_t t,
                                                  uint32_t tag, T z[3][4])
{
    T g[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c) Normals<T>::draw4(seed, job, step, 3u * t + (uint32_t)c, tag, g[c]);
#pragma unroll
    for (int k = 0; k < 12; ++k) z[k % 3][k / 3] = g[k / 4][k % 4];
}

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

}  // namespace sfp
