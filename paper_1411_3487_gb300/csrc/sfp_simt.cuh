// sfp_simt.cuh -- CUDA-core kernels of the mode-space step (FP32 and FP64).
//
// Layout of every per-chain array: [chain][axis][index], index contiguous,
// rows of length M (beads n or modes p).  A "row" j = 3*chain + axis.
#pragma once
#include "sfp_device.cuh"

namespace sfp {

// ---------------------------------------------------------------------------
// Transform GEMM (NT):  Out[j][i] = sum_k In[j][k] * B[i][k]
//   inverse (Eq. e5):  In = R (k = p), B = chi  stored [n][p]  -> Out = u (bonds)
//   forward (Eq. c4):  In = f|z (k = n), B = phi^T stored [p][n] -> Out = DeltaH|Z
// Block tile BM rows x BN cols, K chunk BK; each thread owns TM x TN outputs.
// Any J, Ncols, K (ragged tails are zero-filled).
// ---------------------------------------------------------------------------
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm_nt(const T* __restrict__ In, const T* __restrict__ B, T* __restrict__ Out,
          int J, int Ncols, int K)
{
    constexpr int NT = (BM / TM) * (BN / TN);
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int j0 = blockIdx.y * BM, i0 = blockIdx.x * BN;
    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = T(0);

    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NT) {
            const int row = e / BK, kk = e % BK;
            const int gj = j0 + row, gk = k0 + kk;
            As[kk][row] = (gj < J && gk < K) ? In[(size_t)gj * K + gk] : T(0);
        }
        for (int e = tid; e < BN * BK; e += NT) {
            const int row = e / BK, kk = e % BK;
            const int gi = i0 + row, gk = k0 + kk;
            Bs[kk][row] = (gi < Ncols && gk < K) ? B[(size_t)gi * K + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int x = 0; x < TM; ++x) a[x] = As[kk][ty * TM + x];
#pragma unroll
            for (int y = 0; y < TN; ++y) b[y] = Bs[kk][tx * TN + y];
#pragma unroll
            for (int x = 0; x < TM; ++x)
#pragma unroll
                for (int y = 0; y < TN; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < TM; ++x) {
        const int gj = j0 + ty * TM + x;
        if (gj >= J) continue;
#pragma unroll
        for (int y = 0; y < TN; ++y) {
            const int gi = i0 + tx * TN + y;
            if (gi < Ncols) Out[(size_t)gj * Ncols + gi] = acc[x][y];
        }
    }
}

// ---------------------------------------------------------------------------
// Residual bond force (Eqs. e4, e5, e11), from bond vectors:
//   u_n = sum_p chi_{n,p} R_p (given, n >= 1; slot 0 holds 0),
//   v_n = u_n (1/|u_n| - (1 - 2nu)) for n >= 1, v_0 = 0,
// so that DeltaH_p = sum_n chi_{n,p} v_n (Eq. e11) is the forward transform of
// v with the table chi^T.  The bond form needs no neighbour: each bond's force
// is its own, and the kernel is a stream of 12 B read and 12 B written per
// bond.  One thread per chain and quad of bonds 4t .. 4t+3; threads of a warp
// take consecutive quads, so each axis row moves as one coalesced run of
// float4 (VEC: M % 4 == 0).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void residual_v(const T u[3], bool ok, T c12nu, T v[3])
{
    const T l2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T s = ok ? rsqrt_t<T>(l2) - c12nu : T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = u[a] * s;
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(256)
k_force(const T* __restrict__ ub, T* __restrict__ vb, int C, int M, T c12nu)
{
    const int Q = (M + 3) >> 2;                    // bond quads per chain
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * Q) return;
    const int c = (int)(t / Q), n0 = 4 * (int)(t - (int64_t)c * Q);
    const size_t base = (size_t)c * 3 * M;
    T u[3][4];
    if constexpr (VEC) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float4 x = *reinterpret_cast<const float4*>(ub + base + (size_t)a * M + n0);
            u[a][0] = x.x; u[a][1] = x.y; u[a][2] = x.z; u[a][3] = x.w;
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int i = 0; i < 4; ++i) u[a][i] = n0 + i < M ? ub[base + (size_t)a * M + n0 + i] : T(0);
    }
    T v[3][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T ui[3] = {u[0][i], u[1][i], u[2][i]};
        T vi[3];
        residual_v<T>(ui, n0 + i >= 1 && n0 + i < M, c12nu, vi);
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a][i] = vi[a];
    }
    if constexpr (VEC) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            *reinterpret_cast<float4*>(vb + base + (size_t)a * M + n0) = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (n0 + i < M) vb[base + (size_t)a * M + n0 + i] = v[a][i];
    }
}

// ---------------------------------------------------------------------------
// Bead noise (Eq. b5): z = the bead normals of (seed, job, step, tag 0); normal
// k = 3 n + alpha of a chain and step is value k % 4 of Philox call k / 4.
// With tag 2 the same kernel draws the mode-keyed noise Z (normal 3 p + alpha)
// straight into the mode-space noise buffer.
// One thread per chain and Philox call: its four normals land on two or three
// neighbouring beads, so the threads of a warp write ~43 consecutive beads of
// each axis row.  Bound by the Philox / Box-Muller arithmetic, not by its
// 12 B per bead; it does not depend on the state, so the staged step runs it
// beside the inverse transform.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_noise(T* __restrict__ z, int C, int M, uint32_t seed, const uint32_t* __restrict__ job,
        const int64_t* __restrict__ step, uint32_t tag)
{
    const int K = (3 * M + 3) >> 2;                // Philox calls per chain and step
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * K) return;
    const int c = (int)(t / K), call = (int)(t - (int64_t)c * K);
    T g[4];
    Normals<T>::draw4(seed, job[c], step[c], (uint32_t)call, tag, g);
    T* zc = z + (size_t)c * 3 * M;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int k = 4 * call + e, n = k / 3;
        if (n < M) zc[(size_t)(k - 3 * n) * M + n] = g[e];
    }
}

// ---------------------------------------------------------------------------
// Mode update (Eqs. d3, d6, f2, btum), one thread per (chain, mode), all axes:
//   p >= 1:  R += -dm_p R + h_p DeltaH_p + w_p Z_p ;  R^x += shear g_p R^y(old)
//   p == 0:  r_cm (FP64) += w_0 Z_0 / sqrt(M) ; x_cm += shear dtau y_cm(old);
//            the chain's step counter advances.
// dm_p = 1 - e^{-zeta_p dtau}; written as an increment so FP32 keeps the
// slow modes whose decay factor rounds to 1.
// ---------------------------------------------------------------------------
// V consecutive modes per thread (V = 4: float4 loads and stores, needs
// M % 4 == 0), chains along grid y (grid-stride).  With stop != NULL a chain
// advances only while step < stop, and the step counters are advanced
// afterwards by k_advance_steps (so that no thread of this kernel reads a
// counter that another one changes).
template <typename T, int V>
__device__ __forceinline__ void load_v(const T* p, T (&x)[V])
{
    if constexpr (V == 4 && sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) x[i] = p[i];
    }
}
template <typename T, int V>
__device__ __forceinline__ void store_v(T* p, const T (&x)[V])
{
    if constexpr (V == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) p[i] = x[i];
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(128)
k_mode_update(T* __restrict__ R, const T* __restrict__ DH, const T* __restrict__ ZM,
              double* __restrict__ com, int64_t* __restrict__ step,
              const T* __restrict__ dm, const T* __restrict__ h, const T* __restrict__ w,
              const T* __restrict__ g, const double* __restrict__ shear,
              int C, int M, double w0_cm, double dtau, int* __restrict__ bad,
              const int64_t* __restrict__ stop)
{
    const int p0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (p0 >= M) return;
    for (int c = blockIdx.y * blockDim.y + threadIdx.y; c < C; c += gridDim.y * blockDim.y) {
        // every load of the chain first (one memory round trip), the stop test after
        const size_t b = (size_t)c * 3 * M + p0;
        T r[3][V], y[3][V], zz[3][V], d[V], hh[V], ww[V], gg[V];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            load_v<T, V>(R + b + (size_t)a * M, r[a]);
            load_v<T, V>(DH + b + (size_t)a * M, y[a]);
            load_v<T, V>(ZM + b + (size_t)a * M, zz[a]);
        }
        load_v<T, V>(dm + p0, d);
        load_v<T, V>(h + p0, hh);
        load_v<T, V>(w + p0, ww);
        load_v<T, V>(g + p0, gg);
        const double sh = shear[c];
        const bool run = !stop || step[c] < stop[c];
        double cm[3] = {0.0, 0.0, 0.0};
        if (p0 == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) cm[a] = com[3 * c + a];
        }
        if (!run) continue;
        // the FP64 shear rate is converted only for sheared chains (an integer test
        // of its bits: +0 and -0 mean no shear)
        const bool sheared = (__double_as_longlong(sh) << 1) != 0;
        T o[3][V];
        bool fin = true;
#pragma unroll
        for (int i = 0; i < V; ++i) {
#pragma unroll
            for (int a = 0; a < 3; ++a) o[a][i] = r[a][i] + fma(-d[i], r[a][i], fma(hh[i], y[a][i], ww[i] * zz[a][i]));
#pragma unroll
            for (int a = 0; a < 3; ++a) fin = fin && isfinite(o[a][i]);
        }
        if (sheared) {
            const T shT = (T)sh;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                o[0][i] += shT * gg[i] * r[1][i];
                fin = fin && isfinite(o[0][i]);
            }
        }
        if (p0 == 0) {
            // p = 0: the centre of mass in FP64 (zeta_0 = 0, Eq. d6 limit w_0;
            // w0_cm = w_0 / sqrt(M))
            com[3 * c] = cm[0] + w0_cm * (double)zz[0][0] + sh * dtau * cm[1];
            com[3 * c + 1] = cm[1] + w0_cm * (double)zz[1][0];
            com[3 * c + 2] = cm[2] + w0_cm * (double)zz[2][0];
#pragma unroll
            for (int a = 0; a < 3; ++a) o[a][0] = r[a][0];
            if (!stop) step[c] += 1;
        }
        if (!fin) atomicOr(bad, 1);
#pragma unroll
        for (int a = 0; a < 3; ++a) store_v<T, V>(R + b + (size_t)a * M, o[a]);
    }
}

// ---------------------------------------------------------------------------
// The whole mode-space step (Sec. 4) of one chain per CTA, n_steps per launch,
// on the CUDA cores (the FP64 path): the state stays in shared memory between
// steps, so a small batch (one chain) pays no launch per step.  Per step:
//   thread n (bead):  u_n = sum_p chi_{n,p} R_p (Eq. e5, all three axes from one
//                     pass over chiT[p][n]), v_n = u_n (1/|u_n| - (1 - 2nu)),
//                     v_0 = 0 (Eq. e11); threads c < 3M/4 draw Philox call c of
//                     the step (four bead normals, Eq. b5)
//   thread p (mode):  DeltaH_p = sum_n chi_{n,p} v_n, Z_p = sum_n phi_{n,p} z_n
//                     (Eqs. e11, c4), then R_p += -dm_p R_p + h_p DeltaH_p + w_p Z_p
//                     and the shear term g_p R^y_p on x (Eqs. d3, d6, f2, btum);
//                     p = 0 moves the FP64 centre of mass.
// Tables: chiT [p][n], chi [n][p], phi [n][p] (global, read through L1).  Shared
// memory: R, v, z as [3][M] each.  A chain advances only while step < stop.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_chain_steps(T* __restrict__ Rg, double* __restrict__ com, int64_t* __restrict__ step,
              const int64_t* __restrict__ stop, const uint32_t* __restrict__ job,
              const double* __restrict__ shear, const T* __restrict__ chiT, const T* __restrict__ chi,
              const T* __restrict__ phi, const T* __restrict__ dm, const T* __restrict__ h,
              const T* __restrict__ w, const T* __restrict__ g, int C, int M, T c12nu, double w0_cm,
              double dtau, uint32_t seed, int n_steps, int mode_noise, int* __restrict__ bad)
{
    extern __shared__ unsigned char chain_smem[];
    T* sR = reinterpret_cast<T*>(chain_smem);     // [3][M]
    T* sv = sR + 3 * M;                           // [3][M]
    T* sz = sv + 3 * M;                           // [3][M]
    __shared__ double s_cm[3];
    const int c = blockIdx.x;
    if (c >= C) return;
    T* Rc = Rg + (size_t)c * 3 * M;
    for (int i = threadIdx.x; i < 3 * M; i += blockDim.x) sR[i] = Rc[i];
    if (threadIdx.x < 3) s_cm[threadIdx.x] = com[3 * c + threadIdx.x];
    const uint32_t jb = job[c];
    const double sh = shear[c];
    const T shT = (T)sh;
    const int64_t st0 = step[c];
    const int64_t lim = stop ? stop[c] : INT64_MAX;
    const int n_calls = (3 * M + 3) >> 2;
    bool fin = true;
    __syncthreads();
    int s = 0;
    for (; s < n_steps && st0 + s < lim; ++s) {
        // bond vectors, bond forces, bead normals
        for (int n = threadIdx.x; n < M; n += blockDim.x) {
            T u0 = T(0), u1 = T(0), u2 = T(0);
            for (int p = 1; p < M; ++p) {
                const T x = chiT[(size_t)p * M + n];
                u0 = fma(x, sR[p], u0);
                u1 = fma(x, sR[M + p], u1);
                u2 = fma(x, sR[2 * M + p], u2);
            }
            const T uu[3] = {u0, u1, u2};
            T vv[3];
            residual_v<T>(uu, n >= 1, c12nu, vv);
            sv[n] = vv[0]; sv[M + n] = vv[1]; sv[2 * M + n] = vv[2];
        }
        for (int k = threadIdx.x; k < n_calls; k += blockDim.x) {
            T gq[4];
            Normals<T>::draw4(seed, jb, st0 + s, (uint32_t)k, mode_noise ? 2u : 0u, gq);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int q = 4 * k + e;
                if (q < 3 * M) sz[(q % 3) * M + q / 3] = gq[e];
            }
        }
        __syncthreads();
        // forward transform and update, all three axes of mode p
        for (int p = threadIdx.x; p < M; p += blockDim.x) {
            T d0 = T(0), d1 = T(0), d2 = T(0), z0 = T(0), z1 = T(0), z2 = T(0);
            for (int n = 0; n < M; ++n) {
                const T x = chi[(size_t)n * M + p];
                d0 = fma(x, sv[n], d0);
                d1 = fma(x, sv[M + n], d1);
                d2 = fma(x, sv[2 * M + n], d2);
                if (!mode_noise) {
                    const T f = phi[(size_t)n * M + p];
                    z0 = fma(f, sz[n], z0);
                    z1 = fma(f, sz[M + n], z1);
                    z2 = fma(f, sz[2 * M + n], z2);
                }
            }
            if (mode_noise) {
                // mode-keyed noise: the drawn normals are Z itself
                z0 = sz[p];
                z1 = sz[M + p];
                z2 = sz[2 * M + p];
            }
            if (p == 0) {
                // centre of mass (zeta_0 = 0, Eq. d6 limit; w0_cm = w_0 / sqrt(M)), shear on x
                const double ycm = s_cm[1];
                s_cm[0] += w0_cm * (double)z0 + sh * dtau * ycm;
                s_cm[1] += w0_cm * (double)z1;
                s_cm[2] += w0_cm * (double)z2;
            } else {
                const T r0 = sR[p], r1 = sR[M + p], r2 = sR[2 * M + p];
                const T dd = dm[p], hh = h[p], ww = w[p];
                T o0 = r0 + fma(-dd, r0, fma(hh, d0, ww * z0));
                const T o1 = r1 + fma(-dd, r1, fma(hh, d1, ww * z1));
                const T o2 = r2 + fma(-dd, r2, fma(hh, d2, ww * z2));
                if (shT != T(0)) o0 += shT * g[p] * r1;
                fin = fin && isfinite(o0) && isfinite(o1) && isfinite(o2);
                sR[p] = o0; sR[M + p] = o1; sR[2 * M + p] = o2;
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 3 * M; i += blockDim.x) Rc[i] = (i % M == 0) ? T(0) : sR[i];
    if (threadIdx.x < 3) com[3 * c + threadIdx.x] = s_cm[threadIdx.x];
    if (threadIdx.x == 0) step[c] = st0 + s;
    if (!fin) atomicOr(bad, 1);
}

// ---------------------------------------------------------------------------
// The same FP64 step for a few chains, each on a cluster of G CTAs, so that a
// chain uses the FP64 units of G SMs: CTA r of a chain's cluster owns bonds
// and modes r S .. r S + S - 1 (S = ceil(M / G)) and keeps full copies of R,
// v and z in its shared memory; each owner writes its slice into every CTA of
// the cluster (distributed shared memory).  Per step:
//   owner r:  u_n, v_n of its bonds (Eqs. e5, e11), written to every CTA;
//             every CTA copies the step's bead normals (Eq. b5), drawn for
//             all the steps of the launch beforehand by k_noise_steps, from
//             zpre[s] into its shared memory;
//   cluster barrier;
//   owner r:  DeltaH_p, Z_p of its modes (Eqs. e11, c4), the update of R_p
//             (Eqs. d3, d6, f2, btum; rank 0 the FP64 centre of mass), R_p
//             written to every CTA;
//   cluster barrier.
// Q threads share the sums of one bond or mode (Q a power of 2 within a warp),
// and the groups are dealt round-robin over the four warps: GB300 issues FP64
// arithmetic at a small fraction of the FP32 rate on each SM sub-partition, so
// the work must reach all four of them.  The FP64 Box-Muller of a Philox call
// is a long dependent chain there (~5 us), so the normals come from a separate
// kernel that draws every call of every step at once.  Every CTA
// of a cluster runs the same number of steps (one chain), so the hardware
// cluster barriers always meet.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_cta_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// *p in the shared memory of CTA `rank` of the cluster (p: this CTA's own copy).
__device__ __forceinline__ void st_peer(const double* p, uint32_t rank, double v)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(r), "d"(v) : "memory");
}

template <int G>
__global__ void __launch_bounds__(128)
k_chain_cluster(double* __restrict__ Rg, double* __restrict__ com, int64_t* __restrict__ step,
                const int64_t* __restrict__ stop, const double* __restrict__ shear, const double* __restrict__ chiT,
                const double* __restrict__ chi, const double* __restrict__ phi, const double* __restrict__ dm,
                const double* __restrict__ h, const double* __restrict__ w, const double* __restrict__ g, int C,
                int M, double c12nu, double w0_cm, double dtau, int n_steps, const double* __restrict__ zpre,
                int mode_noise, int* __restrict__ bad)
{
    extern __shared__ unsigned char chain_smem[];
    double* sR = reinterpret_cast<double*>(chain_smem);   // [3][M]
    double* sv = sR + 3 * M;                              // [3][M]
    double* sz = sv + 3 * M;                              // [3][M]
    __shared__ double s_cm[3];
    const uint32_t rank = cluster_cta_rank();
    const int c = blockIdx.x / G;                         // the cluster's chain (c < C: grid = G C)
    const int S = (M + G - 1) / G;
    const int lo = min(M, (int)rank * S), hi = min(M, lo + S), nown = hi - lo;
    int Q = 1;
    while (Q < 32 && 2 * Q * max(nown, 1) <= (int)blockDim.x) Q *= 2;
    const int nwarp = (int)blockDim.x / 32, wid = (int)threadIdx.x / 32, lane = (int)threadIdx.x % 32;
    const int grp = (lane / Q) * nwarp + wid, j = lane % Q, nG = (int)blockDim.x / Q;
    // every thread runs the same passes over the owned bonds / modes (groups past
    // nown compute zeros), so the shuffles always see full warps
    const int passes = (nown + nG - 1) / nG;
    double* Rc = Rg + (size_t)c * 3 * M;
    for (int i = threadIdx.x; i < 3 * M; i += blockDim.x) sR[i] = Rc[i];
    if (threadIdx.x < 3) s_cm[threadIdx.x] = com[3 * c + threadIdx.x];
    const double sh = shear[c];
    const int64_t st0 = step[c];
    const int64_t lim = stop ? stop[c] : INT64_MAX;
    bool fin = true;
    // every CTA of the cluster runs (and has loaded R) before any remote write
    cluster_barrier();
    int s = 0;
    for (; s < n_steps && st0 + s < lim; ++s) {
        const double* zs = zpre + ((size_t)s * C + c) * 3 * M;
        for (int i = threadIdx.x; i < 3 * M; i += blockDim.x) sz[i] = zs[i];
        for (int pass = 0; pass < passes; ++pass) {
            const int gi = pass * nG + grp;
            const bool act = gi < nown;
            const int n = act ? lo + gi : 0;
            double u0 = 0.0, u1 = 0.0, u2 = 0.0;
            for (int p = 1 + j; act && p < M; p += Q) {
                const double x = chiT[(size_t)p * M + n];
                u0 = fma(x, sR[p], u0);
                u1 = fma(x, sR[M + p], u1);
                u2 = fma(x, sR[2 * M + p], u2);
            }
            for (int o = Q / 2; o > 0; o >>= 1) {
                u0 += __shfl_xor_sync(0xffffffffu, u0, o);
                u1 += __shfl_xor_sync(0xffffffffu, u1, o);
                u2 += __shfl_xor_sync(0xffffffffu, u2, o);
            }
            const double uu[3] = {u0, u1, u2};
            double vv[3];
            residual_v<double>(uu, n >= 1, c12nu, vv);
            for (int r = j; act && r < G; r += Q)
                for (int a = 0; a < 3; ++a) st_peer(&sv[a * M + n], (uint32_t)r, vv[a]);
        }
        cluster_barrier();
        for (int pass = 0; pass < passes; ++pass) {
            const int gi = pass * nG + grp;
            const bool act = gi < nown;
            const int p = act ? lo + gi : 0;
            double d0 = 0.0, d1 = 0.0, d2 = 0.0, z0 = 0.0, z1 = 0.0, z2 = 0.0;
            for (int n = j; act && n < M; n += Q) {
                const double x = chi[(size_t)n * M + p];
                d0 = fma(x, sv[n], d0);
                d1 = fma(x, sv[M + n], d1);
                d2 = fma(x, sv[2 * M + n], d2);
                if (!mode_noise) {
                    const double f = phi[(size_t)n * M + p];
                    z0 = fma(f, sz[n], z0);
                    z1 = fma(f, sz[M + n], z1);
                    z2 = fma(f, sz[2 * M + n], z2);
                }
            }
            if (mode_noise && act && j == 0) {
                // mode-keyed noise: Z_p itself (taken once per group)
                z0 = sz[p];
                z1 = sz[M + p];
                z2 = sz[2 * M + p];
            }
            for (int o = Q / 2; o > 0; o >>= 1) {
                d0 += __shfl_xor_sync(0xffffffffu, d0, o);
                d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                d2 += __shfl_xor_sync(0xffffffffu, d2, o);
                z0 += __shfl_xor_sync(0xffffffffu, z0, o);
                z1 += __shfl_xor_sync(0xffffffffu, z1, o);
                z2 += __shfl_xor_sync(0xffffffffu, z2, o);
            }
            if (!act) {
                // a group past the owned modes: nothing to update
            } else if (p == 0) {
                // centre of mass (zeta_0 = 0, Eq. d6 limit; w0_cm = w_0 / sqrt(M)), shear on x
                if (j == 0) {
                    const double ycm = s_cm[1];
                    s_cm[0] += w0_cm * z0 + sh * dtau * ycm;
                    s_cm[1] += w0_cm * z1;
                    s_cm[2] += w0_cm * z2;
                }
            } else {
                const double r0 = sR[p], r1 = sR[M + p], r2 = sR[2 * M + p];
                const double dd = dm[p], hh = h[p], ww = w[p];
                double o0 = r0 + fma(-dd, r0, fma(hh, d0, ww * z0));
                const double o1 = r1 + fma(-dd, r1, fma(hh, d1, ww * z1));
                const double o2 = r2 + fma(-dd, r2, fma(hh, d2, ww * z2));
                if (sh != 0.0) o0 += sh * g[p] * r1;
                fin = fin && isfinite(o0) && isfinite(o1) && isfinite(o2);
                for (int r = j; r < G; r += Q) {
                    st_peer(&sR[p], (uint32_t)r, o0);
                    st_peer(&sR[M + p], (uint32_t)r, o1);
                    st_peer(&sR[2 * M + p], (uint32_t)r, o2);
                }
            }
        }
        cluster_barrier();
    }
    // each CTA writes back its own modes; rank 0 the centre of mass and the counter
    for (int i = threadIdx.x; i < 3 * nown; i += blockDim.x) {
        const int a = i / nown, p = lo + i % nown;
        Rc[a * M + p] = p == 0 ? 0.0 : sR[a * M + p];
    }
    if (rank == 0 && threadIdx.x < 3) com[3 * c + threadIdx.x] = s_cm[threadIdx.x];
    if (rank == 0 && threadIdx.x == 0) step[c] = st0 + s;
    if (!fin) atomicOr(bad, 1);
}

// Bead normals of n_steps consecutive steps for the FP64 cluster path (Eq. b5):
// z[s][c][3][M] = the normals of chain c at step step[c] + s, one thread per
// (step, chain, Philox call); tag 2: the mode-keyed noise Z instead.
__global__ void __launch_bounds__(256)
k_noise_steps(double* __restrict__ z, int C, int M, uint32_t seed, const uint32_t* __restrict__ job,
              const int64_t* __restrict__ step, int n_steps, uint32_t tag)
{
    const int K = (3 * M + 3) >> 2;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_steps * C * K) return;
    const int call = (int)(t % K);
    const int64_t sc = t / K;
    const int c = (int)(sc % C), s = (int)(sc / C);
    double gq[4];
    Normals<double>::draw4(seed, job[c], step[c] + s, (uint32_t)call, tag, gq);
    double* zc = z + ((size_t)s * C + c) * 3 * M;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int k = 4 * call + e, n = k / 3;
        if (n < M) zc[(size_t)(k - 3 * n) * M + n] = gq[e];
    }
}

// step[c] += 1 for chains still below their stop step (after k_mode_update).
__global__ void k_advance_steps(int64_t* __restrict__ step, const int64_t* __restrict__ stop, int C)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C && step[c] < stop[c]) step[c] += 1;
}

// ---------------------------------------------------------------------------
// Equilibrium start, one thread per chain, FP64 (Philox counter (0,0,k,1)):
//   l = l0 + sqrt(T*) L^-T eps   with (I - nu A) = L L^T  (Ld diag, Lo sub-diag)
//   t_1 uniform on the sphere, t_n ~ von Mises-Fisher(t_{n-1}, nu l_{n-1} l_n / T*)
//   r_n = sum_{k<=n} l_k t_k, centroid removed.   out: pos[c][3][M], scratch x[c][M]
// ---------------------------------------------------------------------------
// One chain's equilibrium start (positions p[3][M], scratch x[M]); p and x may
// be global or shared memory.
__device__ void sample_start(double* __restrict__ p, double* __restrict__ x,
                             const double* __restrict__ l0, const double* __restrict__ Ld,
                             const double* __restrict__ Lo, int M, double Tstar, double nu,
                             uint32_t seed, uint32_t job)
{
    const int N = M - 1;
    const uint2 key = make_uint2(seed, job);
    // back substitution L^T x = eps, eps_i is the normal of bond i+1
    for (int i = N - 1; i >= 0; --i) {
        const uint4 wd = philox4x32_10(make_uint4(0u, 0u, (uint32_t)(i + 1), 1u), key);
        double s, co;
        sincospi(2.0 * u01d(wd.y), &s, &co);
        const double eps = sqrt(-2.0 * log(u01d(wd.x))) * co;
        const double nxt = (i + 1 < N) ? Lo[i + 1] * x[i + 1] : 0.0;
        x[i] = (eps - nxt) / Ld[i];
    }
    double t[3];
    {
        const uint4 wd = philox4x32_10(make_uint4(0u, 0u, 0u, 1u), key);
        const double ct = 2.0 * u01d(wd.x) - 1.0;
        const double st = sqrt((1.0 - ct) * (1.0 + ct));
        double sp, cp;
        sincospi(2.0 * u01d(wd.y), &sp, &cp);
        t[0] = st * cp; t[1] = st * sp; t[2] = ct;
    }
    const double sT = sqrt(Tstar);
    double acc[3] = {0.0, 0.0, 0.0}, sum[3] = {0.0, 0.0, 0.0};
    p[0] = p[M] = p[2 * M] = 0.0;
    double lprev = 0.0;
    for (int n = 1; n <= N; ++n) {
        const double ln = l0[n - 1] + sT * x[n - 1];
        if (n >= 2 && Tstar > 0.0) {
            const uint4 wd = philox4x32_10(make_uint4(0u, 0u, (uint32_t)n, 1u), key);
            const double kap = nu * lprev * ln / Tstar;
            const double U = u01d(wd.z);
            const double ct = 1.0 + log(U + (1.0 - U) * exp(-2.0 * kap)) / kap;
            const double st = sqrt(fmax(0.0, (1.0 - ct) * (1.0 + ct)));
            double sp, cp;
            sincospi(2.0 * u01d(wd.w), &sp, &cp);
            // orthonormal pair perpendicular to t (Duff et al., JCGT 2017)
            const double sg = copysign(1.0, t[2]);
            const double a = -1.0 / (sg + t[2]);
            const double bb = t[0] * t[1] * a;
            const double e1[3] = {1.0 + sg * t[0] * t[0] * a, sg * bb, -sg * t[0]};
            const double e2[3] = {bb, sg + t[1] * t[1] * a, -t[1]};
            double tn[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) tn[k] = ct * t[k] + st * (cp * e1[k] + sp * e2[k]);
            const double nn = sqrt(tn[0] * tn[0] + tn[1] * tn[1] + tn[2] * tn[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) t[k] = tn[k] / nn;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc[k] += ln * t[k];
            p[k * M + n] = acc[k];
            sum[k] += acc[k];
        }
        lprev = ln;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double m = sum[k] / M;
        for (int n = 0; n < M; ++n) p[k * M + n] -= m;
    }
}

__global__ void k_equilibrium(double* __restrict__ pos, double* __restrict__ xs,
                              const double* __restrict__ l0, const double* __restrict__ Ld,
                              const double* __restrict__ Lo, int C, int M, double Tstar,
                              double nu, uint32_t seed, const uint32_t* __restrict__ job)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    sample_start(pos + (size_t)c * 3 * M, xs + (size_t)c * M, l0, Ld, Lo, M, Tstar, nu, seed, job[c]);
}

// Serving: start n chains in the slots slot[i] with job key jobv[i], stop step
// stopv[i] and shear rate shv[i] (1/tau).  One block per slot: thread 0 draws the
// equilibrium start into shared memory (3M + M doubles), then the block projects it
// onto the modes R_p = sum_n phi_{n,p} r_n (Eq. c1, p >= 1; phi FP64 [n][p]); the
// centre of mass is at the origin and the step counter 0.
template <typename T>
__global__ void k_init_slots(T* __restrict__ R, double* __restrict__ com, int64_t* __restrict__ step,
                             int64_t* __restrict__ stop, uint32_t* __restrict__ job, double* __restrict__ shear,
                             const int32_t* __restrict__ slot, const uint32_t* __restrict__ jobv,
                             const int64_t* __restrict__ stopv, const double* __restrict__ shv,
                             const double* __restrict__ phi, const double* __restrict__ l0,
                             const double* __restrict__ Ld, const double* __restrict__ Lo,
                             int M, double Tstar, double nu, uint32_t seed)
{
    extern __shared__ double sh_pos[];
    double* xs = sh_pos + 3 * M;
    const int i = blockIdx.x;
    const int c = slot[i];
    if (threadIdx.x == 0) sample_start(sh_pos, xs, l0, Ld, Lo, M, Tstar, nu, seed, jobv[i]);
    __syncthreads();
    T* Rc = R + (size_t)c * 3 * M;
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
        double s[3] = {0.0, 0.0, 0.0};
        if (p > 0)
            for (int n = 0; n < M; ++n) {
                const double f = phi[(size_t)n * M + p];
#pragma unroll
                for (int a = 0; a < 3; ++a) s[a] += f * sh_pos[a * M + n];
            }
#pragma unroll
        for (int a = 0; a < 3; ++a) Rc[(size_t)a * M + p] = (T)s[a];
    }
    if (threadIdx.x == 0) {
        com[3 * c] = com[3 * c + 1] = com[3 * c + 2] = 0.0;
        step[c] = 0;
        stop[c] = stopv[i];
        job[c] = jobv[i];
        shear[c] = shv[i];
    }
}

// Serving: copy the state of slots slot[i] to out[i][3][M] (FP64, R_0 = sqrt(M) r_cm),
// their centres of mass to cm[i][3] and step counters to st[i].
template <typename T>
__global__ void k_gather_slots(const T* __restrict__ R, const double* __restrict__ com,
                               const int64_t* __restrict__ step, const int32_t* __restrict__ slot, int n, int M,
                               double* __restrict__ out, double* __restrict__ cm, int64_t* __restrict__ st)
{
    const int i = blockIdx.x;
    if (i >= n) return;
    const int c = slot[i];
    const double sq = sqrt((double)M);
    for (int e = threadIdx.x; e < 3 * M; e += blockDim.x) {
        const int a = e / M, p = e % M;
        out[(size_t)i * 3 * M + e] = (p == 0) ? com[3 * c + a] * sq : (double)R[(size_t)c * 3 * M + e];
    }
    if (threadIdx.x < 3) cm[3 * i + threadIdx.x] = com[3 * c + threadIdx.x];
    if (threadIdx.x == 0) st[i] = step[c];
}

// ---------------------------------------------------------------------------
// Small conversion kernels.
// ---------------------------------------------------------------------------
// modes (S = FP64 or FP32, packed rows incl. p = 0) -> state R (T, p = 0
// zeroed) + r_cm
template <typename S, typename T>
__global__ void k_load_modes(const S* __restrict__ src, T* __restrict__ R,
                             double* __restrict__ com, int C, int M, double inv_sqrtM)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * 3 * M) return;
    const int p = (int)(t % M);
    const int64_t row = t / M;
    if (p == 0) {
        com[row] = (double)src[t] * inv_sqrtM;
        R[t] = T(0);
    } else {
        R[t] = (T)src[t];
    }
}

// state -> modes (D = FP64 or FP32, R_0 = sqrt(M) r_cm)
template <typename T, typename D>
__global__ void k_store_modes(const T* __restrict__ R, const double* __restrict__ com,
                              D* __restrict__ dst, int C, int M, double sqrtM)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * 3 * M) return;
    const int p = (int)(t % M);
    dst[t] = (p == 0) ? (D)(com[t / M] * sqrtM) : (D)R[t];
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ a, double* __restrict__ b, int64_t n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = (double)a[t];
}

// positions (FP64 scaled, CoM-relative) + CoM -> observables i-iii per chain
__global__ void k_shape(const double* __restrict__ pos, int C, int M, double* __restrict__ out,
                        double d2)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int N = M - 1, mb = (N + 1) / 2, mm = N / 2;
    const double* p = pos + (size_t)c * 3 * M;
    double L2 = 0, u2 = 0, m2 = 0;
    for (int a = 0; a < 3; ++a) {
        const double L = p[a * M + N] - p[a * M];
        const double u = p[a * M + mb] - p[a * M + mb - 1];
        const double m = p[a * M + mm];
        L2 += L * L; u2 += u * u; m2 += m * m;
    }
    out[4 * c + 0] = L2 * d2; out[4 * c + 1] = u2 * d2; out[4 * c + 2] = m2 * d2;
}

__global__ void k_philox_words(uint32_t seed, uint32_t job, int64_t step, uint32_t tag, int n,
                               uint32_t* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 w = philox4x32_10(
        make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)i, tag), make_uint2(seed, job));
    out[4 * i] = w.x; out[4 * i + 1] = w.y; out[4 * i + 2] = w.z; out[4 * i + 3] = w.w;
}

}  // namespace sfp

namespace sfp {

// ---------------------------------------------------------------------------
// Observable sampling (Sec. 5B, observables i-iii), one warp per chain, read
// from the mode state only:
//   L     = r_N - r_0       = sum_p (phi_{N,p} - phi_{0,p}) R_p
//   u_m   (middle bond)     = sum_p chi_{m,p} R_p,          m = ceil(N/2)
//   r_m - r_cm (middle bead)= sum_{p>=1} phi_{m',p} R_p,   m' = floor(N/2)
// tab = [3][M] FP64 coefficient rows for these three sums.  Per chain, adds
// |L|^2, |u_m|^2, |r_m - r_cm|^2 and 1 to shape[c][0..3] and (R_p^a)^2 to
// power[c][a][p] (R_0 = sqrt(M) r_cm).  Displacements over non-overlapping
// windows of lag.v[i] samples (sample index k) of four vectors x: the centre
// of mass (FP64), the middle bead relative to it r_m' - r_cm (observable iii),
// the end-to-end vector L (observable i) and the middle bond u_m (observable
// ii): when k is a multiple of lag.v[i], adds |x - snap_i|^2 and 1 to the
// vector's window sums [c][i][0..1] from the second window edge on and sets
// snap_i = x.  For a stationary X, <X(t).X(0)> = <X^2> - <|X(t) - X(0)|^2> / 2,
// so the windows of L and u_m give their time autocorrelations.  Windows and
// snapshots are [c][kMaxLags][...] whatever lag.n is; win[v] and snp[v] hold
// vector v = 0 (centre of mass), 1 (middle bead), 2 (L), 3 (u_m).
// ---------------------------------------------------------------------------
constexpr int kMaxLags = 8;
struct SampleLags {
    int n;
    int v[kMaxLags];
};

struct SampleWindows {
    double* win[4];    // [C][kMaxLags][2] per vector
    double* snp[4];    // [C][kMaxLags][3] per vector
};

template <typename T>
__global__ void __launch_bounds__(128)
k_sample(const T* __restrict__ R, const double* __restrict__ com, const double* __restrict__ tab,
         int C, int M, double* __restrict__ shape, double* __restrict__ power, SampleWindows wv,
         int64_t k, SampleLags lag)
{
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= C) return;
    const T* Rc = R + (size_t)c * 3 * M;
    double* pw = power + (size_t)c * 3 * M;
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double sqM = sqrt((double)M);
    for (int p = lane; p < M; p += 32) {
        const double cl = tab[p], cu = tab[M + p], cd = tab[2 * M + p];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = (p == 0) ? 0.0 : (double)Rc[(size_t)a * M + p];
            s[a] += cl * x;
            s[3 + a] += cu * x;
            s[6 + a] += cd * x;
            const double xp = (p == 0) ? sqM * com[3 * c + a] : x;
            pw[(size_t)a * M + p] += xp * xp;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
    if (lane != 0) return;
    double* sh = shape + 4 * (size_t)c;
    sh[0] += s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
    sh[1] += s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
    sh[2] += s[6] * s[6] + s[7] * s[7] + s[8] * s[8];
    sh[3] += 1.0;
    const double x[4][3] = {{com[3 * c], com[3 * c + 1], com[3 * c + 2]}, {s[6], s[7], s[8]},
                            {s[0], s[1], s[2]}, {s[3], s[4], s[5]}};
    for (int i = 0; i < lag.n && i < kMaxLags; ++i) {
        if (lag.v[i] <= 0 || k % lag.v[i] != 0) continue;
        const size_t w = (size_t)c * kMaxLags + i;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double* sn = wv.snp[v] + w * 3;
            if (k > 0) {
                double d2 = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double d = x[v][a] - sn[a];
                    d2 += d * d;
                }
                wv.win[v][w * 2] += d2;
                wv.win[v][w * 2 + 1] += 1.0;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) sn[a] = x[v][a];
        }
    }
}

}  // namespace sfp

namespace sfp {

// ---------------------------------------------------------------------------
// Default bead-position Euler scheme (Sec. 3A, Eqs. b3-b5), integrated on the
// bond vectors u_n = r_n - r_{n-1} (n = 1..N; slot 0 unused) with the centre
// of mass in FP64, one block per chain, n_steps steps per launch:
//   e_n = (|u_n| - 1) u_n/|u_n| - nu (u_{n-1} + u_{n+1}),  u_0 = u_{N+1} = 0
//   bead force F_n = e_{n+1} - e_n (e_0 = e_{N+1} = 0), so the bond update is
//   u_n += dtau (e_{n+1} - 2 e_n + e_{n-1}) + a (z_n - z_{n-1}) [+ dtau g u_n^y x]
//   r_cm += a sum_n z_n / M [+ dtau g y_cm x],   a = sqrt(2 T* dtau)
// with z_n the bead normals of the mode-space path (same Philox stream).
// Shared memory: 6 M + 3 values of T (bonds, then noise; e with two zero ends).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_euler_bonds(T* __restrict__ U, double* __restrict__ com, int64_t* __restrict__ step,
                              const uint32_t* __restrict__ job, const double* __restrict__ shear,
                              int C, int M, T dtau, T amp, T nu, uint32_t seed, int n_steps,
                              int* __restrict__ bad)
{
    extern __shared__ unsigned char euler_smem[];
    T* su = reinterpret_cast<T*>(euler_smem);   // [3][M] bonds, later noise
    T* se = su + 3 * M;                          // [3][M+1] e_0 .. e_N (e_0 = 0 stays)
    __shared__ double red[3][32];
    const int c = blockIdx.x;
    if (c >= C) return;
    const int N = M - 1;
    T* Uc = U + (size_t)c * 3 * M;
    const uint32_t jb = job[c];
    const double sh = shear[c];
    int64_t st = step[c];
    bool fin = true;
    for (int s = 0; s < n_steps; ++s, ++st) {
        for (int i = threadIdx.x; i < 3 * M; i += blockDim.x) su[i] = Uc[i];
        __syncthreads();
        // e_n for bonds n = 1..N; e_0 and e_{N+1} are zero
        for (int n = threadIdx.x; n <= N + 1; n += blockDim.x) {
            T e[3] = {T(0), T(0), T(0)};
            if (n >= 1 && n <= N) {
                T u[3], um[3], up[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    u[a] = su[a * M + n];
                    um[a] = n >= 2 ? su[a * M + n - 1] : T(0);
                    up[a] = n + 1 <= N ? su[a * M + n + 1] : T(0);
                }
                const T len = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                const T f = (len - T(1)) / len;
#pragma unroll
                for (int a = 0; a < 3; ++a) e[a] = f * u[a] - nu * (um[a] + up[a]);
            }
            if (n <= N) {
#pragma unroll
                for (int a = 0; a < 3; ++a) se[a * (M + 1) + n] = e[a];
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) se[a * (M + 1) + n] = T(0);
            }
        }
        // bonds stay in registers of the thread that updates them
        __syncthreads();
        T unew[3][4];   // up to 4 bonds per thread (M <= 4 blockDim)
        int k = 0;
        for (int n = threadIdx.x; n < M; n += blockDim.x, ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) unew[a][k] = su[a * M + n];
        __syncthreads();
        // bead noise of this step into su (the bonds are in registers now)
        double zs[3] = {0.0, 0.0, 0.0};
        for (int qd = threadIdx.x; 4 * qd < M; qd += blockDim.x) {
            T g[3][4];
            bead_quad_normals<T>(seed, jb, st, (uint32_t)qd, 0u, g);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int n = 4 * qd + i;
                if (n >= M) break;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    su[a * M + n] = g[a][i];
                    zs[a] += (double)g[a][i];
                }
            }
        }
        // block sum of the noise (centre of mass)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = zs[a];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = v;
        }
        __syncthreads();
        k = 0;
        for (int n = threadIdx.x; n < M; n += blockDim.x, ++k) {
            if (n == 0) continue;
            T o[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T lap = se[a * (M + 1) + n + 1] - T(2) * se[a * (M + 1) + n] + se[a * (M + 1) + n - 1];
                o[a] = unew[a][k] + dtau * lap + amp * (su[a * M + n] - su[a * M + n - 1]);
            }
            o[0] += dtau * (T)sh * unew[1][k];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                fin = fin && isfinite(o[a]);
                Uc[a * M + n] = o[a];
            }
        }
        if (threadIdx.x == 0) {
            double tot[3] = {0.0, 0.0, 0.0};
            for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w)
#pragma unroll
                for (int a = 0; a < 3; ++a) tot[a] += red[a][w];
            double* cm = com + 3 * (size_t)c;
            const double ycm = cm[1];
#pragma unroll
            for (int a = 0; a < 3; ++a) cm[a] += (double)amp * tot[a] / (double)M;
            cm[0] += (double)dtau * sh * ycm;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) step[c] = st;
    if (!fin) atomicOr(bad, 1);
}

}  // namespace sfp
