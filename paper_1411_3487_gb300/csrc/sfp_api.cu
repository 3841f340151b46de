// sfp_api.cu -- host implementation of the C ABI declared in include/sfp.h.
//
// A batch holds one "group" per distinct (n_beads, dtau).  Each group owns
// its FP64-derived tables (Eqs. c8, c9, e9, d3, d6, f2), its chains' state
// R[c][3][M] (p = 0 slot kept at zero; the centre of mass lives in FP64
// r_cm[c][3]), per-chain keys/shear/step counters, and scratch for the
// unfused step: r (beads), f|z (force and noise), DeltaH|Z (mode space).
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/sfp.h"
#include "sfp_fused.h"
#include "sfp_internal.h"
#include "sfp_simt.cuh"
#include "sfp_tc.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(SFP_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));      \
    } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr uint64_t kMagic = 0x3148504653ull;   // "SFPH1"

struct Derived {
    double Tstar, nu, c_ps, d_nm, b, lp_over_a, lambda, kappa;
};

int derive(const sfp_params* p, Derived* d)
{
    if (!p) return fail(SFP_EINVAL, "params is NULL");
    double Tstar, nu;
    if (p->lambda_pN_per_nm > 0.0) {
        if (!(p->kappa_pN_per_nm > 0.0)) return fail(SFP_EINVAL, "kappa must be > 0");
        nu = p->kappa_pN_per_nm / p->lambda_pN_per_nm;
        if (!(nu > 0.0 && nu < 0.5)) return fail(SFP_EINVAL, "nu = kappa/lambda = %g outside (0, 1/2)", nu);
        if (!(p->a_nm > 0.0) || !(p->kT_pN_nm > 0.0))
            return fail(SFP_EINVAL, "a and kT must be > 0 when lambda is given");
        const double dd = p->a_nm * (1.0 - 2.0 * nu);
        Tstar = p->kT_pN_nm / (p->lambda_pN_per_nm * dd * dd);
    } else {
        Tstar = p->T_star;
        nu = p->nu;
        if (!(nu > 0.0 && nu < 0.5)) return fail(SFP_EINVAL, "nu = %g outside (0, 1/2)", nu);
        if (!(Tstar > 0.0)) return fail(SFP_EINVAL, "T_star must be > 0");
    }
    if (!(p->a_nm > 0.0)) return fail(SFP_EINVAL, "a_nm must be > 0");
    double a2xi;
    if (p->a2xi_over_kT_ps > 0.0) {
        a2xi = p->a2xi_over_kT_ps;
    } else {
        if (!(p->xi_kg_per_s > 0.0) || !(p->kT_pN_nm > 0.0))
            return fail(SFP_EINVAL, "xi and kT must be > 0 to compute a^2 xi / kT");
        // (a nm)^2 * xi / (kT pN nm) in ps: 1e-18 m^2 * kg/s / 1e-21 J = 1e3 s -> 1e15 ps
        a2xi = p->a_nm * p->a_nm * p->xi_kg_per_s / p->kT_pN_nm * 1e15;
    }
    const double b = 1.0 / (1.0 - 2.0 * nu);
    d->Tstar = Tstar;
    d->nu = nu;
    d->c_ps = Tstar / (b * b) * a2xi;                       // Eq. g2
    d->d_nm = p->a_nm / b;
    d->b = b;
    d->lp_over_a = b * b * nu / Tstar;                      // Eq. a3
    d->lambda = (p->kT_pN_nm > 0.0) ? p->kT_pN_nm / (Tstar * d->d_nm * d->d_nm) : 0.0;
    d->kappa = nu * d->lambda;
    return SFP_OK;
}

// FP64 tables of one (M, dtau), the closed forms of Eqs. c8, c9, e9, d3, d6, f2
// written for accuracy: 1 - cos t = 2 sin^2(t/2), 1 - e^{-x} = -expm1(-x).
struct Tables {
    std::vector<double> phi, phiT, chi, chiT, dm, h, w, g;   // chi[n][p] = phi[n][p] - phi[n-1][p], chi[0][p] = 0
    double w0;
};

void make_tables(int M, double Tstar, double nu, double dtau, Tables* t)
{
    t->phi.assign((size_t)M * M, 0.0);
    t->phiT.assign((size_t)M * M, 0.0);
    for (int n = 0; n < M; ++n)
        for (int p = 0; p < M; ++p) {
            const double v = (p == 0) ? 1.0 / std::sqrt((double)M)
                                      : std::sqrt(2.0 / M) * std::cos(kPi * p * (n + 0.5) / M);
            t->phi[(size_t)n * M + p] = v;
            t->phiT[(size_t)p * M + n] = v;
        }
    // Eq. e3 (first form): bond vectors u_n = sum_p chi_{n,p} R_p (Eq. e5); row n = 0 is zero.
    t->chi.assign((size_t)M * M, 0.0);
    t->chiT.assign((size_t)M * M, 0.0);
    for (int n = 1; n < M; ++n)
        for (int p = 1; p < M; ++p) {
            t->chi[(size_t)n * M + p] = t->phi[(size_t)n * M + p] - t->phi[(size_t)(n - 1) * M + p];
            t->chiT[(size_t)p * M + n] = t->chi[(size_t)n * M + p];   // DeltaH = chi^T v (Eq. e11)
        }
    t->dm.assign(M, 0.0); t->h.assign(M, 0.0); t->w.assign(M, 0.0); t->g.assign(M, 0.0);
    t->w0 = std::sqrt(2.0 * Tstar * dtau);
    t->g[0] = dtau;
    for (int p = 1; p < M; ++p) {
        const double s2 = std::pow(std::sin(0.5 * kPi * p / M), 2);      // sin^2(theta/2)
        const double zeta = 16.0 * nu * s2 * s2;                           // 4 nu (1 - cos)^2
        const double gap = (1.0 - 2.0 * nu) * 4.0 * s2;                    // zeta^l - zeta
        const double em = -std::expm1(-zeta * dtau);                       // 1 - e^{-zeta dtau}
        t->dm[p] = em;
        t->h[p] = std::exp(-zeta * dtau) * (-std::expm1(-gap * dtau)) / gap;
        t->w[p] = std::sqrt(Tstar * (-std::expm1(-2.0 * zeta * dtau)) / zeta);
        t->g[p] = em / zeta;
    }
}

// Straight-rod ground state (tridiagonal l_n - nu (l_{n-1} + l_{n+1}) = 1) and the
// Cholesky factor of I - nu A.
void rod_tables(int M, double nu, std::vector<double>* l0, std::vector<double>* Ld,
                std::vector<double>* Lo)
{
    const int N = M - 1;
    l0->assign(N, 0.0); Ld->assign(N, 0.0); Lo->assign(N, 0.0);
    std::vector<double> cp(N), dp(N);
    cp[0] = -nu; dp[0] = 1.0;
    for (int i = 1; i < N; ++i) {
        const double den = 1.0 + nu * cp[i - 1];
        cp[i] = -nu / den;
        dp[i] = (1.0 + nu * dp[i - 1]) / den;
    }
    (*l0)[N - 1] = dp[N - 1];
    for (int i = N - 2; i >= 0; --i) (*l0)[i] = dp[i] - cp[i] * (*l0)[i + 1];
    (*Ld)[0] = 1.0;
    for (int i = 1; i < N; ++i) {
        (*Lo)[i] = -nu / (*Ld)[i - 1];
        (*Ld)[i] = std::sqrt(1.0 - (*Lo)[i] * (*Lo)[i]);
    }
}

}  // namespace

int sfp::report(int code, const char* msg) { return fail(code, "%s", msg); }

// Stage timing: events 0..kLastMark of one group-step, around the stages
// inverse, force, noise, forward, update (a fused step records 0 and kLastMark).
constexpr int kMarks = 6, kLastMark = kMarks - 1;

struct Group {
    int M = 0;
    double dtau = 0.0;
    int C = 0;
    std::vector<int> chains;      // indices into the batch's chain list
    Tables tab;
    // device
    void* R = nullptr;            // [C][3][M] state (T)
    double* com = nullptr;        // [C][3]
    uint32_t* job = nullptr;      // [C]
    double* shear = nullptr;      // [C] shear rate in 1/tau
    int64_t* step = nullptr;      // [C]
    int64_t* stop = nullptr;      // [C] a chain advances only while step < stop
    bool limited = false;         // some stop < INT64_MAX (serving pools)
    double* rod = nullptr;        // [3N] ground-state bonds and Cholesky factor (slot starts)
    int32_t* slot_idx = nullptr;  // [C] staging for slot starts
    int32_t* read_idx = nullptr;  // [kGather] staging for slot reads (their own: reads may run beside starts)
    uint32_t* slot_job = nullptr;
    int64_t* slot_stop = nullptr;
    double* slot_shear = nullptr;
    double* gather = nullptr;     // [kGather][3][M] + [kGather][3] + [kGather] FP64 / i64
    void* psiT = nullptr;         // [p][k] = sum_{n >= k} phi_{n,p} (bonds -> modes; Euler path)
    void *chi = nullptr, *chiT = nullptr, *phiT = nullptr, *dm = nullptr, *h = nullptr, *w = nullptr, *g = nullptr;
    double *phi_d = nullptr, *phiT_d = nullptr;   // FP64 copies for conversions
    void* r = nullptr;            // [C][3][M] bond vectors u (slot n = 0 holds 0)
    void* fz = nullptr;           // [2][C][3][M] bond forces v and bead noise z
    void* yz = nullptr;           // [2][C][3][M] DeltaH and Z
    double* stage = nullptr;      // [C][3][M] FP64 staging
    double* stage2 = nullptr;     // [C][3][M] FP64 staging
    sfp::TcPlan* tc = nullptr;    // tensor-core transform plan (SFP_FP32)
    sfp::FusedPlan* fused = nullptr;   // one-kernel step (SFP_FP32 / SFP_MIXED_BF16, M = 64 .. 512)
    bool last_fused = false;      // the most recent step of this group ran fused
    cudaStream_t gs = nullptr;    // this group's stream (batches of several groups)
    cudaEvent_t join = nullptr;
    double* znoise = nullptr;     // FP64 cluster path: bead normals of znoise_steps steps [s][C][3][M]
    int znoise_steps = 0;
    int chain_g = -1;             // FP64 path: CTAs per chain (16, 8, or 0: one CTA per chain); -1 not chosen yet
    cudaStream_t ns = nullptr;    // the staged step's noise kernel, beside the inverse transform
    cudaEvent_t nfork = nullptr, njoin = nullptr;
    // observable sampling (allocated by the first sfp_set_sampling)
    double* obs_tab = nullptr;    // [3][M] rows: phi_N - phi_0, chi_m, phi_m' (p >= 1)
    double* acc_shape = nullptr;  // [C][4]
    double* acc_pow = nullptr;    // [C][3][M]
    double* msd_snap = nullptr;   // [C][kMaxLags][3] centre of mass at the last window edge
    double* msd_acc = nullptr;    // [C][kMaxLags][2]
    double* mid_snap = nullptr;   // [C][kMaxLags][3] r_m' - r_cm at the last window edge
    double* mid_acc = nullptr;    // [C][kMaxLags][2]
    double* e2e_snap = nullptr;   // [C][kMaxLags][3] L at the last window edge
    double* e2e_acc = nullptr;    // [C][kMaxLags][2]
    double* bond_snap = nullptr;  // [C][kMaxLags][3] u_m at the last window edge
    double* bond_acc = nullptr;   // [C][kMaxLags][2]
};

struct sfp_batch {
    Derived dv{};
    int precision = 0;
    uint32_t seed = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0, held = 0;
    int64_t launches = 0;
    bool probed = false;
    int32_t path = SFP_PATH_FUSED;
    int32_t integrator = SFP_INTEGRATOR_MODES;
    // concurrency across length groups and graph replay of step chunks
    cudaStream_t cur = nullptr;        // stream the step path launches on (b->stream or a group's)
    cudaStream_t cap = nullptr;        // capture stream (graphs)
    cudaEvent_t fork = nullptr;
    bool use_graph = false;
    bool grouped = true;               // one launch for the fused groups of all lengths
    int32_t noise = SFP_NOISE_BEADS;   // noise keying of the mode integrator
    int64_t active_limit = -1;         // serving pools: the fused step covers chains [0, limit) (-1: all)
    cudaGraphExec_t graph = nullptr;
    int64_t graph_chunk = 0;
    int64_t graph_launches = 0;        // kernels in one replay
    int C = 0;
    int64_t total_beads = 0;
    std::vector<sfp_chain_desc> desc;
    std::vector<int64_t> off;      // packed offset (elements) of each chain
    std::vector<int> group_of, slot_of;
    std::vector<Group> groups;
    std::vector<void*> allocs;
    int* bad = nullptr;
    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> events;   // pool, kMarks per recorded group-step
    std::vector<char> ev_fused;        // per recorded group-step: events 0 and kLastMark only
    std::vector<int64_t> ev_steps;     // per recorded group-step: steps it covered
    size_t ev_used = 0;
    double stage_us[kMarks] = {0, 0, 0, 0, 0, 0};   // inverse, force, noise, forward, update, step
    int64_t timed_group_steps = 0;
    // observable sampling
    int32_t sample_every = 0;      // 0 = off
    int64_t since_sample = 0;      // steps since the last sample
    int64_t n_samples = 0;         // samples taken since sampling was (re)enabled
    bool sampled = false;          // accumulators exist
    sfp::SampleLags lags{4, {1, 10, 100, 1000}};        // windows of the running sampling
    sfp::SampleLags lags_next{4, {1, 10, 100, 1000}};   // taken by the next sfp_set_sampling
};

namespace {

size_t esize(const sfp_batch* b) { return b->precision == SFP_FP64 ? sizeof(double) : sizeof(float); }

int dalloc(sfp_batch* b, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (b->budget && b->held + bytes > b->budget)
        return fail(SFP_ENOMEM, "HBM budget of %zu bytes exceeded (%zu held, %zu requested)",
                    b->budget, b->held, bytes);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(SFP_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b->held += bytes;
    b->allocs.push_back(*p);
    return SFP_OK;
}

template <typename P> int dalloc_t(sfp_batch* b, P** p, size_t bytes)
{
    void* v = nullptr;
    int rc = dalloc(b, &v, bytes);
    *p = (P*)v;
    return rc;
}

int upload_typed(sfp_batch* b, void* dst, const std::vector<double>& src)
{
    if (b->precision == SFP_FP64) {
        CUDA_TRY(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    } else {
        std::vector<float> f(src.begin(), src.end());
        CUDA_TRY(cudaMemcpyAsync(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
    }
    return SFP_OK;
}

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
int launch_gemm(sfp_batch* b, const T* In, const T* B, T* Out, int J, int Nc, int K)
{
    if constexpr (sizeof(T) == 4) {
        if (Nc >= 128) {
            dim3 grid(nblk(Nc, 128), nblk(J, 128));
            sfp::k_gemm_nt<float, 128, 128, 8, 8, 8><<<grid, 256, 0, b->cur>>>(In, B, Out, J, Nc, K);
        } else {
            dim3 grid(nblk(Nc, 64), nblk(J, 64));
            sfp::k_gemm_nt<float, 64, 64, 8, 4, 4><<<grid, 256, 0, b->cur>>>(In, B, Out, J, Nc, K);
        }
    } else {
        dim3 grid(nblk(Nc, 64), nblk(J, 64));
        sfp::k_gemm_nt<double, 64, 64, 8, 4, 4><<<grid, 256, 0, b->cur>>>(In, B, Out, J, Nc, K);
    }
    b->launches++;
    CUDA_TRY(cudaGetLastError());
    return SFP_OK;
}

// Chains on grid y of the mode update (4 modes per thread when M % 4 == 0).
unsigned chains_y(int C) { return (unsigned)std::min(C, 65535); }

// SFP_TEST_STALL=1 in the environment makes fused launches stall on purpose
// (one bounded wait runs out), to test that a timeout is reported and the
// context stays usable.
int stall_test()
{
    const char* v = std::getenv("SFP_TEST_STALL");
    return v && v[0] == '1' ? 1 : 0;
}

// Launch the staged bond force kernel: one thread per chain and quad of bonds
// (float4 rows when M % 4 == 0).
template <typename T>
cudaError_t launch_force(cudaStream_t st, const T* u, T* v, int C, int M, T c12nu)
{
    const unsigned grid = nblk((int64_t)C * ((M + 3) / 4), 256);
    if (sizeof(T) == 4 && M % 4 == 0)
        sfp::k_force<T, true><<<grid, 256, 0, st>>>(u, v, C, M, c12nu);
    else
        sfp::k_force<T, false><<<grid, 256, 0, st>>>(u, v, C, M, c12nu);
    return cudaGetLastError();
}

// Launch the bead noise kernel: one thread per chain and Philox call.
template <typename T>
cudaError_t launch_noise(cudaStream_t st, T* z, int C, int M, uint32_t seed, const uint32_t* job,
                         const int64_t* step, uint32_t tag = 0u)
{
    const unsigned grid = nblk((int64_t)C * ((3 * M + 3) / 4), 256);
    sfp::k_noise<T><<<grid, 256, 0, st>>>(z, C, M, seed, job, step, tag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mode_update(cudaStream_t st, T* R, const T* DH, const T* ZM, double* com, int64_t* step,
                               const T* dm, const T* h, const T* w, const T* g, const double* shear, int C, int M,
                               double w0, double dtau, int* bad, const int64_t* stop)
{
    // blocks of 128 threads (the kernel's launch bound): a row of modes (V per
    // thread) times as many chains as fill the block
    auto shape = [&](int lanes, dim3& blk, dim3& grid) {
        blk = dim3((unsigned)std::min(lanes, 128), (unsigned)std::max(1, 128 / std::min(lanes, 128)));
        grid = dim3(nblk(lanes, (int)blk.x), chains_y((C + (int)blk.y - 1) / (int)blk.y));
    };
    dim3 blk, grid;
    const double w0_cm = w0 / std::sqrt((double)M);   // noise weight of the centre of mass
    if (sizeof(T) == 4 && M % 4 == 0) {
        shape(M / 4, blk, grid);
        sfp::k_mode_update<T, 4><<<grid, blk, 0, st>>>(R, DH, ZM, com, step, dm, h, w, g, shear, C, M, w0_cm, dtau, bad,
                                                        stop);
    } else {
        shape(M, blk, grid);
        sfp::k_mode_update<T, 1><<<grid, blk, 0, st>>>(R, DH, ZM, com, step, dm, h, w, g, shear, C, M, w0_cm, dtau, bad,
                                                        stop);
    }
    return cudaGetLastError();
}

// Record one event of the current group-step (no-op unless timing is on).
// A fused step records only events 0 and 4.
int mark(sfp_batch* b, int k, bool fused = false, int64_t steps = 1)
{
    if (!b->timing) return SFP_OK;
    if (k == kLastMark) {
        const size_t gs = b->ev_used / kMarks;
        if (b->ev_fused.size() <= gs) b->ev_fused.resize(gs + 1);
        if (b->ev_steps.size() <= gs) b->ev_steps.resize(gs + 1);
        b->ev_fused[gs] = fused;
        b->ev_steps[gs] = steps;
    }
    const size_t idx = b->ev_used + k;
    while (b->events.size() <= idx) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        b->events.push_back(e);
    }
    CUDA_TRY(cudaEventRecord(b->events[idx], b->cur));
    if (k == kLastMark) b->ev_used += kMarks;
    return SFP_OK;
}

// Fold the recorded events into the per-stage totals (synchronises).
int harvest(sfp_batch* b)
{
    if (b->ev_used == 0) return SFP_OK;
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < b->ev_used; i += kMarks) {
        const bool fused = i / kMarks < b->ev_fused.size() && b->ev_fused[i / kMarks];
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, b->events[i], b->events[i + kLastMark]));
        b->stage_us[kLastMark] += 1e3 * ms;
        if (fused) {
            b->stage_us[0] += 1e3 * ms;
        } else {
            for (int k = 0; k < kLastMark; ++k) {
                float mk = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&mk, b->events[i + k], b->events[i + k + 1]));
                b->stage_us[k] += 1e3 * mk;
            }
        }
        b->timed_group_steps += (i / kMarks < b->ev_steps.size()) ? b->ev_steps[i / kMarks] : 1;
    }
    b->ev_used = 0;
    return SFP_OK;
}

// n_steps steps of a group in one launch of the fused kernel (stage timing:
// all of it is recorded as the first stage).
sfp::FusedArgs fused_args(const sfp_batch* b, const Group& g, int64_t n_steps)
{
    sfp::FusedArgs a;
    a.R = (float*)g.R;
    a.com = g.com;
    a.step = g.step;
    a.stop = g.limited ? g.stop : nullptr;
    a.job = g.job;
    a.shear = g.shear;
    a.dm = (const float*)g.dm;
    a.g = (const float*)g.g;
    a.err = b->bad;
    a.C = b->active_limit >= 0 ? (int)std::min<int64_t>(g.C, b->active_limit) : g.C;
    a.c12nu = (float)(1.0 - 2.0 * b->dv.nu);
    a.seed = b->seed;
    a.inv_sqrtM = 1.0 / std::sqrt((double)g.M);
    a.dtau = g.dtau;
    a.n_steps = (int)n_steps;
    a.cpt = sfp::fused_tile(g.fused);
    a.stall_test = stall_test();
    a.zbuf = nullptr;   // the plan's mode-noise buffer and w table, filled in by the launch
    a.w = nullptr;
    return a;
}

int step_group_fused(sfp_batch* b, Group& g, int64_t n_steps)
{
    int rc;
    if ((rc = mark(b, 0))) return rc;
    const sfp::FusedArgs a = fused_args(b, g, n_steps);
    if ((rc = sfp::fused_step(g.fused, a, b->cur))) return rc;
    b->launches++;
    g.last_fused = true;
    return mark(b, kLastMark, true, n_steps);
}

// Groups on the fused step (at most one each of 64, 128, 256 and 512 beads)
// advance together in one launch; their indices, or none if fewer than two
// qualify or grouping is off.
std::vector<size_t> grouped_set(const sfp_batch* b)
{
    std::vector<size_t> out;
    if (!b->grouped || b->timing || b->integrator != SFP_INTEGRATOR_MODES || b->path != SFP_PATH_FUSED ||
        b->noise != SFP_NOISE_BEADS)
        return out;
    bool seen[4] = {false, false, false, false};
    for (size_t i = 0; i < b->groups.size(); ++i) {
        const Group& g = b->groups[i];
        if (!g.fused || !sfp::fused_groupable(g.fused)) continue;
        const int slot = g.M == 512 ? 0 : g.M == 256 ? 1 : g.M == 128 ? 2 : 3;
        if (seen[slot]) continue;
        seen[slot] = true;
        out.push_back(i);
    }
    if (out.size() < 2) out.clear();
    return out;
}

// FP64 groups of up to this many beads take the one-CTA-per-chain kernel on
// SFP_PATH_FUSED (three [3][M] FP64 arrays in shared memory).
constexpr int kChainMaxBeads = 2048;

// The group takes the fused tensor-core step: a fused plan on SFP_PATH_FUSED,
// and with mode-keyed noise a length the fused kernel draws it for.
bool fused_ok(const sfp_batch* b, const Group& g)
{
    if (!g.fused || b->path != SFP_PATH_FUSED) return false;
    return b->noise == SFP_NOISE_BEADS ||
           (sfp::fused_mode_noise_supported(g.M) && b->precision != SFP_MIXED_BF16_2);
}

bool one_launch(const sfp_batch* b, const Group& g)
{
    if (b->path != SFP_PATH_FUSED) return false;
    return fused_ok(b, g) || (b->precision == SFP_FP64 && g.M <= kChainMaxBeads);
}

// n_steps FP64 steps of a group in one launch of k_chain_steps (a CTA per chain,
// state in shared memory between steps); recorded as one fused stage.
// The most bytes of pre-drawn bead normals the FP64 cluster path keeps.
constexpr size_t kNoiseStepBytes = (size_t)32 << 20;

// Launch k_chain_cluster<G> (clusters of G CTAs, one per chain) for k steps.
template <int G>
cudaError_t launch_chain_cluster(sfp_batch* b, Group& g, size_t smem, double c12, double w0cm, int k)
{
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(sfp::k_chain_cluster<G>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(G * g.C));
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->cur;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sfp::k_chain_cluster<G>, (double*)g.R, g.com, g.step,
                              (const int64_t*)(g.limited ? g.stop : nullptr), (const double*)g.shear,
                              (const double*)g.chiT, (const double*)g.chi, (const double*)g.phi_d,
                              (const double*)g.dm, (const double*)g.h, (const double*)g.w, (const double*)g.g, g.C,
                              g.M, c12, w0cm, g.dtau, k, (const double*)g.znoise, b->noise == SFP_NOISE_MODES ? 1 : 0,
                              b->bad);
}

// CTAs per chain for the FP64 cluster path: 16 (a non-portable cluster size)
// when the GPU can place such clusters for this shape, else 8; 0 when the
// batch has too many chains for one cluster each.
int chain_cluster_size(const Group& g, size_t smem, int sms)
{
    if ((int64_t)g.C * 16 <= sms &&
        cudaFuncSetAttribute(sfp::k_chain_cluster<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        (smem <= 48 * 1024 || cudaFuncSetAttribute(sfp::k_chain_cluster<16>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                                  cudaSuccess)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16u * (unsigned)g.C);
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, sfp::k_chain_cluster<16>, &cfg) == cudaSuccess && n >= 1) return 16;
        cudaGetLastError();
    }
    return (int64_t)g.C * 8 <= sms ? 8 : 0;
}

int step_group_chain(sfp_batch* b, Group& g, int64_t n_steps)
{
    int rc;
    if ((rc = mark(b, 0))) return rc;
    const size_t smem = (size_t)9 * g.M * sizeof(double);
    if (smem > 48 * 1024)
        CUDA_TRY(cudaFuncSetAttribute(sfp::k_chain_steps<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    const double c12 = 1.0 - 2.0 * b->dv.nu, w0cm = g.tab.w0 / std::sqrt((double)g.M);
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // few chains: a cluster of CTAs per chain, so that each chain uses several SMs;
    // the bead normals of up to kNoiseStepBytes of steps are drawn beforehand in
    // one kernel (the buffer is allocated on first use, outside stream capture)
    if (g.chain_g < 0) g.chain_g = chain_cluster_size(g, smem, sms);
    const int G = g.chain_g;
    bool cluster = G > 0;
    if (cluster && !g.znoise) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CUDA_TRY(cudaStreamIsCapturing(b->cur, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            const size_t per_step = (size_t)g.C * 3 * g.M * sizeof(double);
            g.znoise_steps = (int)std::max<size_t>(1, std::min<size_t>(1024, kNoiseStepBytes / per_step));
            if ((rc = dalloc_t(b, &g.znoise, per_step * g.znoise_steps))) return rc;
        } else {
            cluster = false;
        }
    }
    if (cluster) {
        for (int64_t done = 0; done < n_steps;) {
            const int k = (int)std::min<int64_t>(g.znoise_steps, n_steps - done);
            const int K = (3 * g.M + 3) / 4;
            sfp::k_noise_steps<<<nblk((int64_t)k * g.C * K, 256), 256, 0, b->cur>>>(
                g.znoise, g.C, g.M, b->seed, g.job, g.step, k, b->noise == SFP_NOISE_MODES ? 2u : 0u);
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(G == 16 ? launch_chain_cluster<16>(b, g, smem, c12, w0cm, k)
                             : launch_chain_cluster<8>(b, g, smem, c12, w0cm, k));
            b->launches += 2;
            done += k;
        }
    } else {
        const int threads = std::min(256, (g.M + 31) / 32 * 32);
        sfp::k_chain_steps<double><<<g.C, threads, smem, b->cur>>>(
            (double*)g.R, g.com, g.step, g.limited ? g.stop : nullptr, g.job, g.shear, (const double*)g.chiT,
            (const double*)g.chi, g.phi_d, (const double*)g.dm, (const double*)g.h, (const double*)g.w,
            (const double*)g.g, g.C, g.M, c12, w0cm, g.dtau, b->seed, (int)n_steps,
            b->noise == SFP_NOISE_MODES ? 1 : 0, b->bad);
        b->launches++;
    }
    CUDA_TRY(cudaGetLastError());
    g.last_fused = true;   // no stage arrays to probe
    return mark(b, kLastMark, true, n_steps);
}

template <typename T>
int step_group(sfp_batch* b, Group& g)
{
    g.last_fused = false;
    const int C = g.C, M = g.M;
    const int64_t n = (int64_t)C * 3 * M;
    T* R = (T*)g.R;
    T* r = (T*)g.r;
    T* fz = (T*)g.fz;
    T* yz = (T*)g.yz;
    int rc;
    if ((rc = mark(b, 0))) return rc;
    // a3: the bead noise depends on the step counters alone, so it runs on a
    // stream of its own beside a1 and a2 (serially while stages are timed)
    const bool side = !b->timing;
    // mode-keyed noise: Z drawn straight into the mode-space buffer, and the
    // forward transform forms DeltaH alone
    const bool mk = b->noise == SFP_NOISE_MODES;
    T* znoise = mk ? yz + n : fz + n;
    const uint32_t ntag = mk ? 2u : 0u;
    if (side) {
        CUDA_TRY(cudaEventRecord(g.nfork, b->cur));
        CUDA_TRY(cudaStreamWaitEvent(g.ns, g.nfork, 0));
        CUDA_TRY(launch_noise<T>(g.ns, znoise, C, M, b->seed, g.job, g.step, ntag));
        CUDA_TRY(cudaEventRecord(g.njoin, g.ns));
        b->launches++;
    }
    // a1: modes -> bond vectors u = chi R  (Eqs. c1, e5; the centre of mass drops out)
    if (g.tc) rc = sfp::tc_transform(g.tc, 0, b->cur);
    else rc = launch_gemm<T>(b, R, (const T*)g.chi, r, 3 * C, M, M);
    if (rc) return rc;
    if (g.tc) b->launches++;
    if ((rc = mark(b, 1))) return rc;
    // a2: residual bond force v (Eq. e11)
    CUDA_TRY(launch_force<T>(b->cur, r, fz, C, M, (T)(1.0 - 2.0 * b->dv.nu)));
    b->launches++;
    if ((rc = mark(b, 2))) return rc;
    if (side) {
        CUDA_TRY(cudaStreamWaitEvent(b->cur, g.njoin, 0));
    } else {
        CUDA_TRY(launch_noise<T>(b->cur, znoise, C, M, b->seed, g.job, g.step, ntag));
        b->launches++;
    }
    if ((rc = mark(b, 3))) return rc;
    // a4: DeltaH = chi^T v (Eq. e11), Z = phi^T z (Eq. c4): the forward transform
    if (g.tc) rc = sfp::tc_transform(g.tc, mk ? 2 : 1, b->cur);
    else if (!(rc = launch_gemm<T>(b, fz, (const T*)g.chiT, yz, 3 * C, M, M)) && !mk)
        rc = launch_gemm<T>(b, fz + n, (const T*)g.phiT, yz + n, 3 * C, M, M);
    if (rc) return rc;
    if (g.tc) b->launches++;
    if ((rc = mark(b, 4))) return rc;
    // a5: mode update (Eqs. d3, d6, f2, btum)
    CUDA_TRY(launch_mode_update<T>(b->cur, R, yz, yz + n, g.com, g.step, (const T*)g.dm, (const T*)g.h,
                                   (const T*)g.w, (const T*)g.g, g.shear, C, M, g.tab.w0, g.dtau, b->bad,
                                   g.limited ? g.stop : nullptr));
    b->launches++;
    if (g.limited) {
        sfp::k_advance_steps<<<nblk(C, 256), 256, 0, b->cur>>>(g.step, g.stop, C);
        b->launches++;
        CUDA_TRY(cudaGetLastError());
    }
    return mark(b, kLastMark);
}

// One sample of observables i-iii, the mode power and the centre-of-mass
// windows for every chain (sample index b->n_samples).
int sample_all(sfp_batch* b)
{
    for (auto& g : b->groups) {
        const unsigned grid = nblk(g.C, 4);
        const sfp::SampleWindows wv{{g.msd_acc, g.mid_acc, g.e2e_acc, g.bond_acc},
                                    {g.msd_snap, g.mid_snap, g.e2e_snap, g.bond_snap}};
        if (b->precision == SFP_FP64)
            sfp::k_sample<double><<<grid, 128, 0, b->stream>>>((const double*)g.R, g.com, g.obs_tab, g.C, g.M,
                                                               g.acc_shape, g.acc_pow, wv, b->n_samples, b->lags);
        else
            sfp::k_sample<float><<<grid, 128, 0, b->stream>>>((const float*)g.R, g.com, g.obs_tab, g.C, g.M,
                                                              g.acc_shape, g.acc_pow, wv, b->n_samples, b->lags);
        b->launches++;
        CUDA_TRY(cudaGetLastError());
    }
    b->n_samples++;
    b->since_sample = 0;
    return SFP_OK;
}

// n_steps of the default bead-position Euler scheme (Eqs. b3-b5) for a group:
// bonds u = chi R (Eq. e5), k_euler_bonds on the bonds and the FP64 centre of
// mass, then back to modes R_p = sum_n phi_{n,p} r_n = sum_k psi_{k,p} u_k with
// psi_{k,p} = sum_{n >= k} phi_{n,p} (p >= 1; constant shifts drop out).
template <typename T>
int step_group_euler(sfp_batch* b, Group& g, int64_t n_steps)
{
    const int C = g.C, M = g.M;
    int rc;
    if (!g.psiT) {
        std::vector<double> psi((size_t)M * M, 0.0);
        for (int p = 1; p < M; ++p) {
            double acc = 0.0;
            for (int k = M - 1; k >= 1; --k) {
                acc += g.tab.phi[(size_t)k * M + p];
                psi[(size_t)p * M + k] = acc;
            }
        }
        if ((rc = dalloc(b, &g.psiT, (size_t)M * M * sizeof(T))) || (rc = upload_typed(b, g.psiT, psi))) return rc;
    }
    if ((rc = mark(b, 0))) return rc;
    if (g.tc) {
        if ((rc = sfp::tc_transform(g.tc, 0, b->cur))) return rc;
    } else if ((rc = launch_gemm<T>(b, (const T*)g.R, (const T*)g.chi, (T*)g.r, 3 * C, M, M))) {
        return rc;
    }
    const int threads = std::min(1024, (M + 31) / 32 * 32);
    if ((M + threads - 1) / threads > 4) return fail(SFP_ENOTSUP, "the Euler path supports up to 4096 beads");
    const size_t smem = (size_t)(6 * M + 3) * sizeof(T);
    if (smem > 48 * 1024)
        CUDA_TRY(cudaFuncSetAttribute(sfp::k_euler_bonds<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int64_t s0 = 0; s0 < n_steps; s0 += 1024) {
        const int k = (int)std::min<int64_t>(1024, n_steps - s0);
        sfp::k_euler_bonds<T><<<C, threads, smem, b->cur>>>((T*)g.r, g.com, g.step, g.job, g.shear, C, M,
                                                                (T)g.dtau, (T)std::sqrt(2.0 * b->dv.Tstar * g.dtau),
                                                                (T)b->dv.nu, b->seed, k, b->bad);
        CUDA_TRY(cudaGetLastError());
        b->launches++;
    }
    if ((rc = launch_gemm<T>(b, (const T*)g.r, (const T*)g.psiT, (T*)g.R, 3 * C, M, M))) return rc;
    g.last_fused = true;   // no stage arrays to probe
    return mark(b, kLastMark, true, n_steps);
}

constexpr int64_t kMaxFusedSteps = 1024;   // steps per fused launch

// The launches of one chunk of steps for every group.  With several groups
// (and no stage timing) each group runs on its own stream, forked from and
// joined back into `base`, so groups of different lengths share the GPU.
int issue_chunk(sfp_batch* b, int64_t chunk, cudaStream_t base)
{
    const bool conc = b->groups.size() > 1 && !b->timing;
    if (conc) {
        CUDA_TRY(cudaEventRecord(b->fork, base));
        for (auto& g : b->groups) CUDA_TRY(cudaStreamWaitEvent(g.gs, b->fork, 0));
    }
    int rc = SFP_OK;
    // the groups with the most transform work (C M^2) are issued first, so that
    // the longest launch starts first when the groups share the GPU
    std::vector<size_t> order(b->groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        const Group &gx = b->groups[x], &gy = b->groups[y];
        return (double)gx.C * gx.M * gx.M > (double)gy.C * gy.M * gy.M;
    });
    const std::vector<size_t> grp = grouped_set(b);
    bool grp_done = false;
    for (size_t gi : order) {
        Group& g = b->groups[gi];
        b->cur = conc ? g.gs : base;
        if (std::find(grp.begin(), grp.end(), gi) != grp.end()) {
            // the grouped launch, issued in the place of the heaviest of its groups
            if (grp_done) continue;
            grp_done = true;
            std::vector<sfp::FusedPlan*> plans;
            std::vector<sfp::FusedArgs> args;
            for (size_t k : grp) {
                plans.push_back(b->groups[k].fused);
                args.push_back(fused_args(b, b->groups[k], chunk));
                b->groups[k].last_fused = true;
            }
            if ((rc = sfp::fused_step_grouped(plans.data(), args.data(), (int)plans.size(), b->cur))) break;
            b->launches++;
            continue;
        }
        if (b->integrator == SFP_INTEGRATOR_EULER) {
            rc = (b->precision == SFP_FP64) ? step_group_euler<double>(b, g, chunk)
                                            : step_group_euler<float>(b, g, chunk);
        } else if (fused_ok(b, g)) {
            rc = step_group_fused(b, g, chunk);
        } else if (one_launch(b, g)) {
            rc = step_group_chain(b, g, chunk);
        } else {
            for (int64_t k = 0; k < chunk && rc == SFP_OK; ++k)
                rc = (b->precision == SFP_FP64) ? step_group<double>(b, g) : step_group<float>(b, g);
        }
        if (rc) break;
    }
    if (conc) {
        for (auto& g : b->groups) {
            const cudaError_t e1 = cudaEventRecord(g.join, g.gs);
            const cudaError_t e2 = cudaStreamWaitEvent(base, g.join, 0);
            if (!rc && (e1 != cudaSuccess || e2 != cudaSuccess)) rc = fail(SFP_ECUDA, "stream join failed");
        }
    }
    b->cur = b->stream;
    return rc;
}

void drop_graph(sfp_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_chunk = 0;
}

// One chunk through a CUDA graph: captured on the batch's capture stream the
// first time a chunk of this length is issued, then replayed on its stream.
int graph_chunk(sfp_batch* b, int64_t chunk)
{
    if (!b->graph || b->graph_chunk != chunk) {
        drop_graph(b);
        CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = b->launches;
        const int rc = issue_chunk(b, chunk, b->cap);
        b->graph_launches = b->launches - l0;
        b->launches = l0;                 // captured, not run: counted per replay below
        cudaGraph_t gph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &gph);
        if (rc) {
            if (gph) cudaGraphDestroy(gph);
            return rc;
        }
        if (e != cudaSuccess) return fail(SFP_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        const cudaError_t ei = cudaGraphInstantiate(&b->graph, gph, 0);
        cudaGraphDestroy(gph);
        if (ei != cudaSuccess) {
            b->graph = nullptr;
            return fail(SFP_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
        }
        b->graph_chunk = chunk;
    }
    CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
    b->launches += b->graph_launches;
    return SFP_OK;
}

int step_all(sfp_batch* b, int64_t n_steps)
{
    bool staged = false;
    for (auto& g : b->groups) staged = staged || !one_launch(b, g);
    const bool graphs = b->use_graph && !b->timing && b->integrator == SFP_INTEGRATOR_MODES;
    for (int64_t s = 0; s < n_steps;) {
        // steps up to the next observable sample: one launch per fused group,
        // one launch per stage and step for the others
        int64_t chunk = std::min<int64_t>(n_steps - s, kMaxFusedSteps);
        if (graphs && staged) chunk = std::min<int64_t>(chunk, 64);   // bounded graph size
        if (b->sample_every > 0) chunk = std::min<int64_t>(chunk, b->sample_every - b->since_sample);
        const int rc = graphs ? graph_chunk(b, chunk) : issue_chunk(b, chunk, b->stream);
        if (rc) return rc;
        s += chunk;
        if (b->sample_every > 0 && (b->since_sample += chunk) == b->sample_every) {
            const int rc = sample_all(b);
            if (rc) return rc;
        }
        if (b->timing && b->ev_used >= 4000) {
            const int rc = harvest(b);
            if (rc) return rc;
        }
    }
    if (n_steps > 0) b->probed = true;
    return SFP_OK;
}

// Modes (S = double or float, device-readable, [C][3][M] incl. p = 0) -> state
template <typename S>
int load_modes_dev(sfp_batch* b, Group& g, const S* src)
{
    const int64_t n = (int64_t)g.C * 3 * g.M;
    const double inv = 1.0 / std::sqrt((double)g.M);
    if (b->precision == SFP_FP64)
        sfp::k_load_modes<S, double><<<nblk(n, 256), 256, 0, b->stream>>>(src, (double*)g.R, g.com, g.C, g.M, inv);
    else
        sfp::k_load_modes<S, float><<<nblk(n, 256), 256, 0, b->stream>>>(src, (float*)g.R, g.com, g.C, g.M, inv);
    CUDA_TRY(cudaGetLastError());
    return SFP_OK;
}

// State -> modes (D = double or float, device-writable, [C][3][M], R_0 = sqrt(M) r_cm)
template <typename D>
int store_modes_dev(sfp_batch* b, Group& g, D* dst)
{
    const int64_t n = (int64_t)g.C * 3 * g.M;
    const double sq = std::sqrt((double)g.M);
    if (b->precision == SFP_FP64)
        sfp::k_store_modes<double, D><<<nblk(n, 256), 256, 0, b->stream>>>((const double*)g.R, g.com, dst, g.C, g.M, sq);
    else
        sfp::k_store_modes<float, D><<<nblk(n, 256), 256, 0, b->stream>>>((const float*)g.R, g.com, dst, g.C, g.M, sq);
    CUDA_TRY(cudaGetLastError());
    return SFP_OK;
}

int to_double(sfp_batch* b, const void* src, double* dst, int64_t n)
{
    if (b->precision == SFP_FP64)
        CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    else {
        sfp::k_to_double<float><<<nblk(n, 256), 256, 0, b->stream>>>((const float*)src, dst, n);
        CUDA_TRY(cudaGetLastError());
    }
    return SFP_OK;
}

// The device address of a page-locked host buffer that the GPU can reach
// (NVLink-C2C / PCIe loads and stores), or nullptr for pageable memory.  The
// conversion kernels then read or write the caller's buffer directly instead
// of staging it with a copy.
const void* mapped_host(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Gather host packed [3][M_c] blocks of one group into a contiguous host array.
template <typename E>
void gather_group(const sfp_batch* b, const Group& g, const E* packed, std::vector<E>& out)
{
    const size_t blk = (size_t)3 * g.M;
    out.resize((size_t)g.C * blk);
    for (int i = 0; i < g.C; ++i)
        std::memcpy(out.data() + i * blk, packed + b->off[g.chains[i]], blk * sizeof(E));
}

template <typename E>
void scatter_group(const sfp_batch* b, const Group& g, const std::vector<E>& in, E* packed)
{
    const size_t blk = (size_t)3 * g.M;
    for (int i = 0; i < g.C; ++i)
        std::memcpy(packed + b->off[g.chains[i]], in.data() + i * blk, blk * sizeof(E));
}

// CoM-relative bead positions (FP64, scaled) of a group into g.stage2
int positions_dev(sfp_batch* b, Group& g)
{
    const int64_t n = (int64_t)g.C * 3 * g.M;
    int rc = to_double(b, g.R, g.stage, n);
    if (rc) return rc;
    return launch_gemm<double>(b, g.stage, g.phi_d, g.stage2, 3 * g.C, g.M, g.M);
}

int destroy_impl(sfp_batch* b)
{
    if (!b) return SFP_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    for (auto& g : b->groups) {
        if (g.gs) cudaStreamSynchronize(g.gs);
        if (g.tc) sfp::tc_destroy(g.tc);
        if (g.fused) sfp::fused_destroy(g.fused);
        if (g.ns) cudaStreamSynchronize(g.ns);
        if (g.gs) cudaStreamDestroy(g.gs);
        if (g.join) cudaEventDestroy(g.join);
        if (g.ns) cudaStreamDestroy(g.ns);
        if (g.nfork) cudaEventDestroy(g.nfork);
        if (g.njoin) cudaEventDestroy(g.njoin);
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
    return SFP_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free step: scratch and tables in one file-scope device array.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[SFP_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  The host-side
// name is only a stand-in and must never reach a kernel.  The address is looked
// up on every call (a host-side query, not a stream operation), so it stays
// right after the device's primary context has been reset and recreated.
int noalloc_scratch(unsigned char** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(SFP_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    *out = (unsigned char*)p;
    return SFP_OK;
}

// Tables of Eqs. c8, e3, c9, e9, d3, d6, f2 computed on the device in FP64, stored FP32.
__device__ __forceinline__ double phi_dev(int M, int n, int p)
{
    return (p == 0) ? rsqrt((double)M) : sqrt(2.0 / M) * cospi((double)p * (n + 0.5) / M);
}
__global__ void k_noalloc_tables(float* chi, float* chiT, float* phiT, float* dm, float* h, float* w, float* g,
                                 int M, double Tstar, double nu, double dtau)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (int64_t)M * M) {
        const int n = (int)(t / M), p = (int)(t % M);
        phiT[(size_t)p * M + n] = (float)phi_dev(M, n, p);
        const float c = (n == 0 || p == 0) ? 0.f : (float)(phi_dev(M, n, p) - phi_dev(M, n - 1, p));
        chi[(size_t)n * M + p] = c;
        chiT[(size_t)p * M + n] = c;
    }
    if (t < M) {
        const int p = (int)t;
        if (p == 0) {
            dm[0] = 0.f; h[0] = 0.f; w[0] = (float)sqrt(2.0 * Tstar * dtau); g[0] = (float)dtau;
        } else {
            const double sn = sinpi(0.5 * p / M);
            const double s2 = sn * sn;
            const double zeta = 16.0 * nu * s2 * s2;
            const double gap = (1.0 - 2.0 * nu) * 4.0 * s2;
            const double em = -expm1(-zeta * dtau);
            dm[p] = (float)em;
            h[p] = (float)(exp(-zeta * dtau) * (-expm1(-gap * dtau)) / gap);
            w[p] = (float)sqrt(Tstar * (-expm1(-2.0 * zeta * dtau)) / zeta);
            g[p] = (float)(em / zeta);
        }
    }
}

// Per-call state: step counters, keys, shear, p = 0 entries cleared.
__global__ void k_noalloc_prep(float* R, int64_t* step, uint32_t* job, double* shear, int* bad, int C, int M,
                               int64_t step0, uint32_t job0, double shear_tau)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) *bad = 0;
    if (c >= C) return;
    step[c] = step0;
    job[c] = job0 + (uint32_t)c;
    shear[c] = shear_tau;
    for (int a = 0; a < 3; ++a) R[((size_t)c * 3 + a) * M] = 0.f;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
cudaError_t gemm_on(cudaStream_t st, const T* In, const T* B, T* Out, int J, int Nc, int K)
{
    if (Nc >= 128) {
        dim3 grid(nblk(Nc, 128), nblk(J, 128));
        sfp::k_gemm_nt<T, 128, 128, 8, 8, 8><<<grid, 256, 0, st>>>(In, B, Out, J, Nc, K);
    } else {
        dim3 grid(nblk(Nc, 64), nblk(J, 64));
        sfp::k_gemm_nt<T, 64, 64, 8, 4, 4><<<grid, 256, 0, st>>>(In, B, Out, J, Nc, K);
    }
    return cudaGetLastError();
}

// sfp_set_modes body for host element type S (double or float).
template <typename S>
int set_modes_impl(sfp_batch* b, const S* host, size_t n)
{
    if (!b || !host) return fail(SFP_EINVAL, "NULL argument");
    if (n < (size_t)(3 * b->total_beads)) return fail(SFP_EINVAL, "need %lld values", (long long)(3 * b->total_beads));
    std::vector<S> tmp;
    for (auto& g : b->groups) {
        const S* dev = b->groups.size() == 1 ? (const S*)mapped_host(host) : nullptr;
        if (dev) {   // one group, page-locked caller buffer: the kernel reads it directly
            int rc = load_modes_dev(b, g, dev);
            if (rc) return rc;
            CUDA_TRY(cudaStreamSynchronize(b->stream));
            continue;
        }
        S* stage = (S*)g.stage;   // [C][3][M] doubles: room for either type
        if (b->groups.size() == 1) {   // packed order is the group order: copy straight from the caller
            CUDA_TRY(cudaMemcpyAsync(stage, host, (size_t)g.C * 3 * g.M * sizeof(S), cudaMemcpyHostToDevice, b->stream));
        } else {
            gather_group(b, g, host, tmp);
            CUDA_TRY(cudaMemcpyAsync(stage, tmp.data(), tmp.size() * sizeof(S), cudaMemcpyHostToDevice, b->stream));
        }
        int rc = load_modes_dev(b, g, (const S*)stage);
        if (rc) return rc;
        CUDA_TRY(cudaStreamSynchronize(b->stream));
    }
    b->probed = false;
    return SFP_OK;
}

// SFP_OBS_MODES / SFP_OBS_MODES_F32 of one group into the caller's packed
// array.  With one group and a page-locked caller buffer the kernel writes it
// directly and returns without waiting (sfp_observe's error-word read waits for
// the stream).
template <typename D>
int observe_modes(sfp_batch* b, Group& g, D* host_out, std::vector<D>& tmp)
{
    const int64_t n = (int64_t)g.C * 3 * g.M;
    D* direct = b->groups.size() == 1 ? (D*)mapped_host(host_out) : nullptr;
    D* dst = direct ? direct : (D*)g.stage;
    int rc = store_modes_dev(b, g, dst);
    if (rc || direct) return rc;
    if (b->groups.size() == 1) {
        CUDA_TRY(cudaMemcpyAsync(host_out, dst, n * sizeof(D), cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
    } else {
        tmp.resize(n);
        CUDA_TRY(cudaMemcpyAsync(tmp.data(), dst, n * sizeof(D), cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        scatter_group(b, g, tmp, host_out);
    }
    return SFP_OK;
}

}  // namespace

extern "C" {

int sfp_params_dsdna(sfp_params* p)
{
    if (!p) return fail(SFP_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof *p);
    p->T_star = 0.034;
    p->nu = 0.35;
    p->a_nm = 0.33;
    p->xi_kg_per_s = 1.91e-12;
    p->kT_pN_nm = 4.089;
    p->a2xi_over_kT_ps = 52.0;
    return SFP_OK;
}

int sfp_derive(const sfp_params* p, double out[8])
{
    if (!out) return fail(SFP_EINVAL, "out is NULL");
    Derived d;
    const int rc = derive(p, &d);
    if (rc) return rc;
    out[0] = d.Tstar; out[1] = d.nu; out[2] = d.c_ps; out[3] = d.d_nm;
    out[4] = d.b; out[5] = d.lp_over_a; out[6] = d.lambda; out[7] = d.kappa;
    return SFP_OK;
}

const char* sfp_last_error(void) { return g_err.c_str(); }

int sfp_create(const sfp_params* params, const sfp_chain_desc* chains, int32_t n_chains,
               uint64_t seed, int32_t precision, void* cuda_stream, size_t hbm_budget_bytes,
               sfp_batch** out)
{
    if (!out) return fail(SFP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!chains || n_chains <= 0) return fail(SFP_EINVAL, "need n_chains > 0 and a chain array");
    if (seed >> 32) return fail(SFP_EINVAL, "seed must be < 2^32");
    if (precision != SFP_FP32 && precision != SFP_FP64 && precision != SFP_FP32_SIMT && precision != SFP_MIXED_BF16 &&
        precision != SFP_MIXED_BF16_2)
        return fail(SFP_EINVAL, "unknown precision %d", precision);
    Derived dv;
    int rc = derive(params, &dv);
    if (rc) return rc;
    sfp_batch* b = new sfp_batch();
    b->dv = dv;
    b->precision = precision;
    b->seed = (uint32_t)seed;
    b->stream = (cudaStream_t)cuda_stream;
    b->budget = hbm_budget_bytes;
    b->C = n_chains;
    b->desc.assign(chains, chains + n_chains);
    b->off.resize(n_chains);
    b->group_of.resize(n_chains);
    b->slot_of.resize(n_chains);
    std::map<std::pair<int, double>, int> gidx;
    int64_t acc = 0;
    for (int i = 0; i < n_chains; ++i) {
        const sfp_chain_desc& d = chains[i];
        if (d.n_beads < 3 || d.n_beads > 4096) { delete b; return fail(SFP_EINVAL, "chain %d: n_beads %d outside 3..4096", i, d.n_beads); }
        if (d.reserved != 0) { delete b; return fail(SFP_EINVAL, "chain %d: reserved must be 0", i); }
        if (d.job_id >> 32) { delete b; return fail(SFP_EINVAL, "chain %d: job_id must be < 2^32", i); }
        const double dtau = d.dtau > 0.0 ? d.dtau : d.dt_ps / dv.c_ps;
        if (!(dtau > 0.0) || !std::isfinite(dtau)) { delete b; return fail(SFP_EINVAL, "chain %d: step must be > 0", i); }
        if (!std::isfinite(d.shear_rate_per_s)) { delete b; return fail(SFP_EINVAL, "chain %d: shear rate not finite", i); }
        b->off[i] = acc;
        acc += 3 * (int64_t)d.n_beads;
        const auto key = std::make_pair((int)d.n_beads, dtau);
        auto it = gidx.find(key);
        int gi;
        if (it == gidx.end()) {
            gi = (int)b->groups.size();
            gidx[key] = gi;
            b->groups.emplace_back();
            b->groups.back().M = d.n_beads;
            b->groups.back().dtau = dtau;
        } else {
            gi = it->second;
        }
        b->group_of[i] = gi;
        b->slot_of[i] = (int)b->groups[gi].chains.size();
        b->groups[gi].chains.push_back(i);
    }
    b->total_beads = acc / 3;
    const size_t es = (precision == SFP_FP64) ? 8 : 4;
    if ((rc = dalloc_t(b, &b->bad, sizeof(int)))) { destroy_impl(b); return rc; }
    for (auto& g : b->groups) {
        const int M = g.M;
        g.C = (int)g.chains.size();
        const size_t n = (size_t)g.C * 3 * M;
        make_tables(M, dv.Tstar, dv.nu, g.dtau, &g.tab);
        if ((rc = dalloc(b, &g.R, n * es)) || (rc = dalloc_t(b, &g.com, (size_t)g.C * 3 * 8)) ||
            (rc = dalloc_t(b, &g.job, (size_t)g.C * 4)) || (rc = dalloc_t(b, &g.shear, (size_t)g.C * 8)) ||
            (rc = dalloc_t(b, &g.step, (size_t)g.C * 8)) || (rc = dalloc_t(b, &g.stop, (size_t)g.C * 8)) ||
            (rc = dalloc(b, &g.chi, (size_t)M * M * es)) || (rc = dalloc(b, &g.chiT, (size_t)M * M * es)) ||
            (rc = dalloc(b, &g.phiT, (size_t)M * M * es)) || (rc = dalloc(b, &g.dm, M * es)) ||
            (rc = dalloc(b, &g.h, M * es)) || (rc = dalloc(b, &g.w, M * es)) || (rc = dalloc(b, &g.g, M * es)) ||
            (rc = dalloc_t(b, &g.phi_d, (size_t)M * M * 8)) || (rc = dalloc_t(b, &g.phiT_d, (size_t)M * M * 8)) ||
            (rc = dalloc(b, &g.r, n * es)) || (rc = dalloc(b, &g.fz, 2 * n * es)) ||
            (rc = dalloc(b, &g.yz, 2 * n * es)) || (rc = dalloc_t(b, &g.stage, n * 8)) ||
            (rc = dalloc_t(b, &g.stage2, n * 8))) {
            destroy_impl(b);
            return rc;
        }
        if ((rc = upload_typed(b, g.chi, g.tab.chi)) || (rc = upload_typed(b, g.chiT, g.tab.chiT)) ||
            (rc = upload_typed(b, g.phiT, g.tab.phiT)) ||
            (rc = upload_typed(b, g.dm, g.tab.dm)) || (rc = upload_typed(b, g.h, g.tab.h)) ||
            (rc = upload_typed(b, g.w, g.tab.w)) || (rc = upload_typed(b, g.g, g.tab.g))) {
            destroy_impl(b);
            return rc;
        }
        std::vector<uint32_t> jobs(g.C);
        std::vector<double> sh(g.C);
        std::vector<int64_t> st(g.C, 0), nostop(g.C, INT64_MAX);
        for (int i = 0; i < g.C; ++i) {
            const sfp_chain_desc& d = chains[g.chains[i]];
            jobs[i] = (uint32_t)d.job_id;
            sh[i] = d.shear_rate_per_s * dv.c_ps * 1e-12;   // 1/s -> 1/tau
        }
        // Straight ground-state rod along x, centre of mass at the origin.
        std::vector<double> l0, Ld, Lo;
        rod_tables(M, dv.nu, &l0, &Ld, &Lo);
        std::vector<double> rod((size_t)3 * M, 0.0), Rrod((size_t)3 * M, 0.0);
        for (int k = 1; k < M; ++k) rod[k] = rod[k - 1] + l0[k - 1];
        double cm = 0.0;
        for (int k = 0; k < M; ++k) cm += rod[k];
        cm /= M;
        for (int k = 0; k < M; ++k) rod[k] -= cm;
        for (int p = 1; p < M; ++p) {
            double s = 0.0;
            for (int k = 0; k < M; ++k) s += rod[k] * g.tab.phi[(size_t)k * M + p];
            Rrod[p] = s;
        }
        std::vector<double> init(n);
        for (int i = 0; i < g.C; ++i) std::memcpy(init.data() + (size_t)i * 3 * M, Rrod.data(), 3 * M * sizeof(double));
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.job, jobs.data(), g.C * 4, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.shear, sh.data(), g.C * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.step, st.data(), g.C * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.stop, nostop.data(), g.C * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.phi_d, g.tab.phi.data(), (size_t)M * M * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.phiT_d, g.tab.phiT.data(), (size_t)M * M * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.stage, init.data(), n * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->bad, 0, sizeof(int), b->stream);
        if (e != cudaSuccess) { destroy_impl(b); return fail(SFP_ECUDA, "upload failed: %s", cudaGetErrorString(e)); }
        if ((rc = load_modes_dev(b, g, g.stage))) { destroy_impl(b); return rc; }
        e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) { destroy_impl(b); return fail(SFP_ECUDA, "create: %s", cudaGetErrorString(e)); }
        const bool bf16 = precision == SFP_MIXED_BF16 || precision == SFP_MIXED_BF16_2;
        const bool two = precision == SFP_MIXED_BF16_2;
        if ((precision == SFP_FP32 || bf16) && sfp::tc_supported(M)) {
            rc = sfp::tc_create(&g.tc, M, 3 * g.C, g.tab.chi.data(), g.tab.chiT.data(), g.tab.phiT.data(),
                                (const float*)g.R,
                                (float*)g.r, (const float*)g.fz, (float*)g.yz, b->bad, b->stream,
                                bf16, two);
            if (rc) { destroy_impl(b); return rc; }
        }
        if ((precision == SFP_FP32 || bf16) && sfp::fused_supported(M)) {
            std::vector<double> w = g.tab.w;
            w[0] = g.tab.w0;
            rc = sfp::fused_create(&g.fused, M, g.C, g.tab.chi.data(), g.tab.phi.data(), g.tab.h.data(), w.data(),
                                   (float*)g.R, b->stream, bf16, two);
            if (rc) { destroy_impl(b); return rc; }
        }
        if (precision == SFP_FP64 && M <= kChainMaxBeads) {
            // the FP64 chain path: a cluster of CTAs per chain for few chains, with
            // its buffer of pre-drawn normals allocated here, outside any capture
            int dev = 0, sms = 0;
            e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) { destroy_impl(b); return fail(SFP_ECUDA, "create: %s", cudaGetErrorString(e)); }
            g.chain_g = chain_cluster_size(g, (size_t)9 * M * sizeof(double), sms);
            if (g.chain_g > 0) {
                const size_t per_step = (size_t)g.C * 3 * M * sizeof(double);
                g.znoise_steps = (int)std::max<size_t>(1, std::min<size_t>(1024, kNoiseStepBytes / per_step));
                if ((rc = dalloc_t(b, &g.znoise, per_step * g.znoise_steps))) { destroy_impl(b); return rc; }
            }
        }
        b->held += sfp::tc_bytes(g.tc) + sfp::fused_bytes(g.fused);
        if (b->budget && b->held > b->budget) {
            const size_t held = b->held;
            destroy_impl(b);
            return fail(SFP_ENOMEM, "HBM budget of %zu bytes exceeded (%zu needed)", hbm_budget_bytes, held);
        }
    }
    // Lengths that share one grouped launch (at most one group each of 64, 128,
    // 256 and 512 beads): chains per tile chosen for all of them together, not
    // for each group as if it had the GPU to itself.  If tiles of 40 chains (the
    // fewest MMAs per chain) take more than one wave of the SMs, 40 (the
    // autotuner's choice on 8192 mixed chains); else the smallest tiles that
    // still fit one wave.
    {
        std::vector<size_t> cand;
        bool seen[4] = {false, false, false, false};
        for (size_t i = 0; i < b->groups.size(); ++i) {
            const Group& g = b->groups[i];
            if (!g.fused) continue;
            const int slot = g.M == 512 ? 0 : g.M == 256 ? 1 : g.M == 128 ? 2 : 3;
            if (seen[slot]) continue;
            seen[slot] = true;
            cand.push_back(i);
        }
        int dev = 0, sms = 0;
        if (cand.size() >= 2 && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
            auto ctas = [&](int cpt) {
                int64_t n = 0;
                for (size_t i : cand) {
                    const Group& g = b->groups[i];
                    n += (int64_t)((g.C + cpt - 1) / cpt) * (g.M == 512 ? 2 : 1);
                }
                return n;
            };
            int best = 40;
            if (ctas(40) <= sms)
                for (int cpt = 4; cpt <= 40; cpt += 4)
                    if (ctas(cpt) <= sms) {
                        best = cpt;
                        break;
                    }
            for (size_t i : cand)
                if ((rc = sfp::fused_set_tile(b->groups[i].fused, best))) { destroy_impl(b); return rc; }
        }
    }
    b->cur = b->stream;
    {
        cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (auto& g : b->groups) {
            if (e != cudaSuccess) break;
            e = cudaStreamCreateWithFlags(&g.ns, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.nfork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.njoin, cudaEventDisableTiming);
            if (e != cudaSuccess || b->groups.size() < 2) continue;
            e = cudaStreamCreateWithFlags(&g.gs, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) { destroy_impl(b); return fail(SFP_ECUDA, "stream creation failed: %s", cudaGetErrorString(e)); }
    }
    *out = b;
    return SFP_OK;
}

int sfp_destroy(sfp_batch* b) { return destroy_impl(b); }

int sfp_step(sfp_batch* b, int64_t n_steps)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (n_steps < 0) return fail(SFP_EINVAL, "n_steps < 0");
    return step_all(b, n_steps);
}

int sfp_set_step(sfp_batch* b, int64_t step)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (step < 0) return fail(SFP_EINVAL, "step < 0");
    for (auto& g : b->groups) {
        std::vector<int64_t> st(g.C, step);
        CUDA_TRY(cudaMemcpyAsync(g.step, st.data(), g.C * 8, cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
    }
    return SFP_OK;
}

int sfp_set_modes(sfp_batch* b, const double* host, size_t n_doubles)
{
    return set_modes_impl(b, host, n_doubles);
}

int sfp_set_modes_f32(sfp_batch* b, const float* host, size_t n_floats)
{
    return set_modes_impl(b, host, n_floats);
}

int sfp_set_positions(sfp_batch* b, const double* host, size_t n_doubles)
{
    if (!b || !host) return fail(SFP_EINVAL, "NULL argument");
    if (n_doubles < (size_t)(3 * b->total_beads)) return fail(SFP_EINVAL, "need %lld doubles", (long long)(3 * b->total_beads));
    std::vector<double> tmp;
    const double inv_d = 1.0 / b->dv.d_nm;
    for (auto& g : b->groups) {
        gather_group(b, g, host, tmp);
        for (auto& x : tmp) x *= inv_d;
        CUDA_TRY(cudaMemcpyAsync(g.stage2, tmp.data(), tmp.size() * 8, cudaMemcpyHostToDevice, b->stream));
        int rc = launch_gemm<double>(b, g.stage2, g.phiT_d, g.stage, 3 * g.C, g.M, g.M);
        if (rc) return rc;
        if ((rc = load_modes_dev(b, g, g.stage))) return rc;
        CUDA_TRY(cudaStreamSynchronize(b->stream));
    }
    b->probed = false;
    return SFP_OK;
}

int sfp_init_equilibrium(sfp_batch* b, int64_t burn_in_steps)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (burn_in_steps < 0) return fail(SFP_EINVAL, "burn_in_steps < 0");
    for (auto& g : b->groups) {
        std::vector<double> l0, Ld, Lo;
        rod_tables(g.M, b->dv.nu, &l0, &Ld, &Lo);
        std::vector<double> all;
        all.insert(all.end(), l0.begin(), l0.end());
        all.insert(all.end(), Ld.begin(), Ld.end());
        all.insert(all.end(), Lo.begin(), Lo.end());
        const int N = g.M - 1;
        // l0 | Ld | Lo live in the head of stage2's tail-free region: use yz scratch
        double* tabs = nullptr;
        double* xs = nullptr;
        CUDA_TRY(cudaMalloc(&tabs, all.size() * 8));
        cudaError_t e = cudaMalloc(&xs, (size_t)g.C * g.M * 8);
        if (e != cudaSuccess) { cudaFree(tabs); return fail(SFP_ENOMEM, "init scratch: %s", cudaGetErrorString(e)); }
        e = cudaMemcpyAsync(tabs, all.data(), all.size() * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) {
            sfp::k_equilibrium<<<nblk(g.C, 64), 64, 0, b->stream>>>(g.stage2, xs, tabs, tabs + N, tabs + 2 * N,
                                                                   g.C, g.M, b->dv.Tstar, b->dv.nu, b->seed, g.job);
            e = cudaGetLastError();
        }
        int rc = SFP_OK;
        if (e == cudaSuccess) rc = launch_gemm<double>(b, g.stage2, g.phiT_d, g.stage, 3 * g.C, g.M, g.M);
        if (e == cudaSuccess && !rc) rc = load_modes_dev(b, g, g.stage);
        if (e == cudaSuccess && !rc) e = cudaMemsetAsync(g.com, 0, (size_t)g.C * 3 * 8, b->stream);
        if (e == cudaSuccess && !rc) e = cudaMemsetAsync(g.step, 0, (size_t)g.C * 8, b->stream);
        if (e == cudaSuccess && !rc) e = cudaStreamSynchronize(b->stream);
        cudaFree(tabs);
        cudaFree(xs);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(SFP_ECUDA, "init_equilibrium: %s", cudaGetErrorString(e));
    }
    b->probed = false;
    return step_all(b, burn_in_steps);
}

int sfp_observe(sfp_batch* b, int32_t what, void* host_out, size_t bytes)
{
    if (!b || !host_out) return fail(SFP_EINVAL, "NULL argument");
    const size_t packed = (size_t)3 * b->total_beads * sizeof(double);
    size_t need = 0;
    switch (what) {
        case SFP_OBS_MODES: case SFP_OBS_POSITIONS: need = packed; break;
        case SFP_OBS_MODES_F32: need = packed / 2; break;
        case SFP_OBS_COM: need = (size_t)b->C * 3 * 8; break;
        case SFP_OBS_STEP: need = (size_t)b->C * 8; break;
        case SFP_OBS_SHAPE: need = (size_t)b->C * 4 * 8; break;
        case SFP_OBS_ACCUM: need = (size_t)b->C * 4 * 8; break;
        case SFP_OBS_MODE_POWER: case SFP_OBS_MODE_VAR: need = packed; break;
        case SFP_OBS_COM_MSD: case SFP_OBS_MID_MSD: case SFP_OBS_E2E_MSD: case SFP_OBS_BOND_MSD:
            need = (size_t)b->C * b->lags.n * 2 * 8;
            break;
        case SFP_OBS_E2E2_MEAN: need = (size_t)b->C * 8; break;
        default: return fail(SFP_EINVAL, "unknown observable %d", what);
    }
    if ((what == SFP_OBS_ACCUM || what == SFP_OBS_MODE_POWER || what == SFP_OBS_COM_MSD || what == SFP_OBS_MID_MSD ||
         what == SFP_OBS_E2E_MSD || what == SFP_OBS_BOND_MSD || what == SFP_OBS_E2E2_MEAN ||
         what == SFP_OBS_MODE_VAR) && !b->sampled)
        return fail(SFP_EINVAL, "observable %d needs sfp_set_sampling first", what);
    if (bytes < need) return fail(SFP_EINVAL, "buffer too small: need %zu bytes", need);
    std::vector<double> tmp;
    std::vector<float> tmp32;
    for (auto& g : b->groups) {
        const int64_t n = (int64_t)g.C * 3 * g.M;
        if (what == SFP_OBS_MODES) {
            int rc = observe_modes(b, g, (double*)host_out, tmp);
            if (rc) return rc;
        } else if (what == SFP_OBS_MODES_F32) {
            int rc = observe_modes(b, g, (float*)host_out, tmp32);
            if (rc) return rc;
        } else if (what == SFP_OBS_POSITIONS || what == SFP_OBS_SHAPE) {
            int rc = positions_dev(b, g);
            if (rc) return rc;
            if (what == SFP_OBS_SHAPE) {
                std::vector<double> sh((size_t)g.C * 4);
                sfp::k_shape<<<nblk(g.C, 128), 128, 0, b->stream>>>(g.stage2, g.C, g.M, g.stage, b->dv.d_nm * b->dv.d_nm);
                CUDA_TRY(cudaGetLastError());
                CUDA_TRY(cudaMemcpyAsync(sh.data(), g.stage, sh.size() * 8, cudaMemcpyDeviceToHost, b->stream));
                std::vector<int64_t> st(g.C);
                CUDA_TRY(cudaMemcpyAsync(st.data(), g.step, g.C * 8, cudaMemcpyDeviceToHost, b->stream));
                CUDA_TRY(cudaStreamSynchronize(b->stream));
                for (int i = 0; i < g.C; ++i) {
                    double* o = (double*)host_out + 4 * (size_t)g.chains[i];
                    o[0] = sh[4 * i]; o[1] = sh[4 * i + 1]; o[2] = sh[4 * i + 2];
                    o[3] = (double)st[i] * g.dtau * b->dv.c_ps;
                }
            } else {
                tmp.resize(n);
                std::vector<double> cm((size_t)g.C * 3);
                CUDA_TRY(cudaMemcpyAsync(tmp.data(), g.stage2, n * 8, cudaMemcpyDeviceToHost, b->stream));
                CUDA_TRY(cudaMemcpyAsync(cm.data(), g.com, cm.size() * 8, cudaMemcpyDeviceToHost, b->stream));
                CUDA_TRY(cudaStreamSynchronize(b->stream));
                const double dnm = b->dv.d_nm;
                for (int i = 0; i < g.C; ++i)
                    for (int a = 0; a < 3; ++a)
                        for (int k = 0; k < g.M; ++k) {
                            double& x = tmp[((size_t)i * 3 + a) * g.M + k];
                            x = (x + cm[3 * i + a]) * dnm;
                        }
                scatter_group(b, g, tmp, (double*)host_out);
            }
        } else if (what == SFP_OBS_COM) {
            std::vector<double> cm((size_t)g.C * 3);
            CUDA_TRY(cudaMemcpyAsync(cm.data(), g.com, cm.size() * 8, cudaMemcpyDeviceToHost, b->stream));
            CUDA_TRY(cudaStreamSynchronize(b->stream));
            for (int i = 0; i < g.C; ++i)
                for (int a = 0; a < 3; ++a) ((double*)host_out)[3 * (size_t)g.chains[i] + a] = cm[3 * i + a] * b->dv.d_nm;
        } else if (what == SFP_OBS_ACCUM || what == SFP_OBS_E2E2_MEAN) {
            std::vector<double> a((size_t)g.C * 4);
            CUDA_TRY(cudaMemcpyAsync(a.data(), g.acc_shape, a.size() * 8, cudaMemcpyDeviceToHost, b->stream));
            CUDA_TRY(cudaStreamSynchronize(b->stream));
            const double d2 = b->dv.d_nm * b->dv.d_nm;
            double* o = (double*)host_out;
            for (int i = 0; i < g.C; ++i) {
                const double* ai = a.data() + 4 * (size_t)i;
                if (what == SFP_OBS_E2E2_MEAN) {
                    o[g.chains[i]] = ai[3] > 0.0 ? ai[0] / ai[3] * d2 : 0.0;
                } else {
                    // sums in nm^2; the count as it is
                    for (int k = 0; k < 4; ++k) o[(size_t)4 * g.chains[i] + k] = ai[k] * (k == 3 ? 1.0 : d2);
                }
            }
        } else if (what == SFP_OBS_COM_MSD || what == SFP_OBS_MID_MSD || what == SFP_OBS_E2E_MSD ||
                   what == SFP_OBS_BOND_MSD) {
            const int L = b->lags.n;
            std::vector<double> a((size_t)g.C * sfp::kMaxLags * 2);
            const double* src = what == SFP_OBS_COM_MSD ? g.msd_acc : what == SFP_OBS_MID_MSD ? g.mid_acc
                              : what == SFP_OBS_E2E_MSD ? g.e2e_acc : g.bond_acc;
            CUDA_TRY(cudaMemcpyAsync(a.data(), src, a.size() * 8, cudaMemcpyDeviceToHost, b->stream));
            CUDA_TRY(cudaStreamSynchronize(b->stream));
            const double d2 = b->dv.d_nm * b->dv.d_nm;
            for (int i = 0; i < g.C; ++i)
                for (int l = 0; l < L; ++l) {
                    const double* w = a.data() + ((size_t)i * sfp::kMaxLags + l) * 2;
                    double* o = (double*)host_out + ((size_t)g.chains[i] * L + l) * 2;
                    o[0] = w[0] * d2;   // sum in nm^2
                    o[1] = w[1];        // windows
                }
        } else if (what == SFP_OBS_MODE_POWER || what == SFP_OBS_MODE_VAR) {
            tmp.resize(n);
            CUDA_TRY(cudaMemcpyAsync(tmp.data(), g.acc_pow, n * 8, cudaMemcpyDeviceToHost, b->stream));
            if (what == SFP_OBS_MODE_VAR) {
                std::vector<double> a((size_t)g.C * 4);
                CUDA_TRY(cudaMemcpyAsync(a.data(), g.acc_shape, a.size() * 8, cudaMemcpyDeviceToHost, b->stream));
                CUDA_TRY(cudaStreamSynchronize(b->stream));
                for (int i = 0; i < g.C; ++i) {
                    const double cnt = a[4 * (size_t)i + 3];
                    for (int k = 0; k < 3 * g.M; ++k) tmp[(size_t)i * 3 * g.M + k] = cnt > 0.0 ? tmp[(size_t)i * 3 * g.M + k] / cnt : 0.0;
                }
            }
            CUDA_TRY(cudaStreamSynchronize(b->stream));
            scatter_group(b, g, tmp, (double*)host_out);
        } else if (what == SFP_OBS_STEP) {
            std::vector<int64_t> st(g.C);
            CUDA_TRY(cudaMemcpyAsync(st.data(), g.step, g.C * 8, cudaMemcpyDeviceToHost, b->stream));
            CUDA_TRY(cudaStreamSynchronize(b->stream));
            for (int i = 0; i < g.C; ++i) ((int64_t*)host_out)[g.chains[i]] = st[i];
        }
    }
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, b->bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (bad & 4) return fail(SFP_ECUDA, "a 512-bead fused step ran without its two-CTA cluster");
    if (bad & 2) return fail(SFP_ETIMEDOUT, "a tensor-core pipeline wait timed out");
    if (bad & 1) return fail(SFP_ENONFINITE, "a chain's state became non-finite");
    return SFP_OK;
}

int sfp_probe(sfp_batch* b, int32_t what, void* host_out, size_t bytes)
{
    if (!b || !host_out) return fail(SFP_EINVAL, "NULL argument");
    if (what < SFP_PROBE_BONDS || what > SFP_PROBE_ZMODE) return fail(SFP_EINVAL, "unknown probe %d", what);
    if (!b->probed) return fail(SFP_EINVAL, "no step has run since the state was set");
    for (const auto& g : b->groups)
        if (g.last_fused) return fail(SFP_EINVAL, "the last step ran fused; probes need SFP_PATH_STAGED");
    const size_t need = (size_t)3 * b->total_beads * 8;
    if (bytes < need) return fail(SFP_EINVAL, "buffer too small: need %zu bytes", need);
    std::vector<double> tmp;
    const size_t es = esize(b);
    for (auto& g : b->groups) {
        const int64_t n = (int64_t)g.C * 3 * g.M;
        const char* src = nullptr;
        switch (what) {
            case SFP_PROBE_BONDS: src = (const char*)g.r; break;
            case SFP_PROBE_FORCE: src = (const char*)g.fz; break;
            case SFP_PROBE_NOISE: src = (const char*)g.fz + n * es; break;
            case SFP_PROBE_DH: src = (const char*)g.yz; break;
            case SFP_PROBE_ZMODE: src = (const char*)g.yz + n * es; break;
        }
        int rc = to_double(b, src, g.stage, n);
        if (rc) return rc;
        tmp.resize(n);
        CUDA_TRY(cudaMemcpyAsync(tmp.data(), g.stage, n * 8, cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        scatter_group(b, g, tmp, (double*)host_out);
    }
    return SFP_OK;
}

int sfp_save(sfp_batch* b, void* host_buf, size_t bytes, size_t* needed)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    const size_t need = 4 * 8 + (size_t)3 * b->total_beads * 8 + (size_t)b->C * 3 * 8 + (size_t)b->C * 8;
    if (needed) *needed = need;
    if (!host_buf) return SFP_OK;
    if (bytes < need) return fail(SFP_EINVAL, "buffer too small: need %zu bytes", need);
    uint64_t* hdr = (uint64_t*)host_buf;
    hdr[0] = kMagic; hdr[1] = (uint64_t)b->C; hdr[2] = (uint64_t)b->total_beads; hdr[3] = (uint64_t)b->precision;
    double* modes = (double*)(hdr + 4);
    double* com = modes + 3 * b->total_beads;
    int64_t* st = (int64_t*)(com + 3 * (size_t)b->C);
    std::vector<double> tmp;
    for (auto& g : b->groups) {
        const int64_t n = (int64_t)g.C * 3 * g.M;
        int rc = to_double(b, g.R, g.stage, n);
        if (rc) return rc;
        tmp.resize(n);
        std::vector<double> cm((size_t)g.C * 3);
        std::vector<int64_t> s(g.C);
        CUDA_TRY(cudaMemcpyAsync(tmp.data(), g.stage, n * 8, cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaMemcpyAsync(cm.data(), g.com, cm.size() * 8, cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaMemcpyAsync(s.data(), g.step, g.C * 8, cudaMemcpyDeviceToHost, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        scatter_group(b, g, tmp, modes);
        for (int i = 0; i < g.C; ++i) {
            const int c = g.chains[i];
            for (int a = 0; a < 3; ++a) com[3 * (size_t)c + a] = cm[3 * i + a];
            st[c] = s[i];
        }
    }
    return SFP_OK;
}

int sfp_load(sfp_batch* b, const void* host_buf, size_t bytes)
{
    if (!b || !host_buf) return fail(SFP_EINVAL, "NULL argument");
    const size_t need = 4 * 8 + (size_t)3 * b->total_beads * 8 + (size_t)b->C * 3 * 8 + (size_t)b->C * 8;
    if (bytes < need) return fail(SFP_EINVAL, "checkpoint too small: need %zu bytes", need);
    const uint64_t* hdr = (const uint64_t*)host_buf;
    if (hdr[0] != kMagic || hdr[1] != (uint64_t)b->C || hdr[2] != (uint64_t)b->total_beads ||
        hdr[3] != (uint64_t)b->precision)
        return fail(SFP_EINVAL, "checkpoint does not match this batch");
    const double* modes = (const double*)(hdr + 4);
    const double* com = modes + 3 * b->total_beads;
    const int64_t* st = (const int64_t*)(com + 3 * (size_t)b->C);
    std::vector<double> tmp;
    for (auto& g : b->groups) {
        gather_group(b, g, modes, tmp);
        CUDA_TRY(cudaMemcpyAsync(g.stage, tmp.data(), tmp.size() * 8, cudaMemcpyHostToDevice, b->stream));
        int rc = load_modes_dev(b, g, g.stage);
        if (rc) return rc;
        std::vector<double> cm((size_t)g.C * 3);
        std::vector<int64_t> s(g.C);
        for (int i = 0; i < g.C; ++i) {
            const int c = g.chains[i];
            for (int a = 0; a < 3; ++a) cm[3 * i + a] = com[3 * (size_t)c + a];
            s[i] = st[c];
        }
        CUDA_TRY(cudaMemcpyAsync(g.com, cm.data(), cm.size() * 8, cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(cudaMemcpyAsync(g.step, s.data(), g.C * 8, cudaMemcpyHostToDevice, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
    }
    b->probed = false;
    return SFP_OK;
}

int sfp_info(const sfp_batch* b, int64_t out[4])
{
    if (!b || !out) return fail(SFP_EINVAL, "NULL argument");
    out[0] = b->C; out[1] = b->total_beads; out[2] = (int64_t)b->held; out[3] = b->launches;
    return SFP_OK;
}

int sfp_stage_timing(sfp_batch* b, int32_t enable)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    int rc = harvest(b);
    if (rc) return rc;
    b->timing = enable != 0;
    const size_t want = 5 * b->groups.size() * 64;
    while (b->timing && b->events.size() < want) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        b->events.push_back(e);
    }
    for (double& x : b->stage_us) x = 0.0;
    b->timed_group_steps = 0;
    return SFP_OK;
}

int sfp_stage_times(sfp_batch* b, double out_us[6], int64_t* n_group_steps)
{
    if (!b || !out_us) return fail(SFP_EINVAL, "NULL argument");
    int rc = harvest(b);
    if (rc) return rc;
    for (int k = 0; k < kMarks; ++k) out_us[k] = b->stage_us[k];
    if (n_group_steps) *n_group_steps = b->timed_group_steps;
    return SFP_OK;
}

int sfp_set_path(sfp_batch* b, int32_t path)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (path != SFP_PATH_FUSED && path != SFP_PATH_STAGED) return fail(SFP_EINVAL, "unknown path %d", path);
    if (b->path != path) drop_graph(b);
    b->path = path;
    return SFP_OK;
}

int sfp_set_noise(sfp_batch* b, int32_t keying)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (keying != SFP_NOISE_BEADS && keying != SFP_NOISE_MODES) return fail(SFP_EINVAL, "unknown noise keying %d", keying);
    if (keying == SFP_NOISE_MODES) {
        for (auto& g : b->groups) {
            if (!g.fused || !sfp::fused_mode_noise_supported(g.M) || b->precision == SFP_MIXED_BF16_2) continue;
            const size_t before = sfp::fused_bytes(g.fused);
            int rc = sfp::fused_set_mode_noise(g.fused, true);
            if (rc) return fail(rc, "%s", sfp_last_error());
            b->held += sfp::fused_bytes(g.fused) - before;
        }
    } else {
        for (auto& g : b->groups)
            if (g.fused) sfp::fused_set_mode_noise(g.fused, false);
    }
    if (b->noise != keying) drop_graph(b);
    b->noise = keying;
    return SFP_OK;
}

int sfp_set_grouped(sfp_batch* b, int32_t enable)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (b->grouped != (enable != 0)) drop_graph(b);
    b->grouped = enable != 0;
    return SFP_OK;
}

int sfp_set_graph(sfp_batch* b, int32_t enable)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (!enable) drop_graph(b);
    b->use_graph = enable != 0;
    return SFP_OK;
}

int sfp_autotune(sfp_batch* b, int32_t trial_steps, int32_t* chains_per_tile)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (trial_steps < 1) return fail(SFP_EINVAL, "trial_steps must be >= 1");
    const size_t G = b->groups.size();
    if (chains_per_tile)
        for (size_t i = 0; i < G; ++i) chains_per_tile[i] = b->groups[i].fused ? sfp::fused_tile(b->groups[i].fused) : 0;
    if (b->path != SFP_PATH_FUSED || b->integrator != SFP_INTEGRATOR_MODES || b->timing) return SFP_OK;
    std::vector<size_t> fg;
    for (size_t i = 0; i < G; ++i)
        if (fused_ok(b, b->groups[i])) fg.push_back(i);
    if (fg.empty()) return SFP_OK;
    int dev = 0, sms = 148;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // save every group's dynamic state; each trial starts from it again
    struct Saved { void* R = nullptr; double* com = nullptr; int64_t* step = nullptr; };
    std::vector<Saved> sv(G);
    auto release = [&]() {
        for (auto& x : sv) { cudaFree(x.R); cudaFree(x.com); cudaFree(x.step); }
    };
    const size_t es = esize(b);
    for (size_t i = 0; i < G; ++i) {
        const Group& g = b->groups[i];
        const size_t n = (size_t)g.C * 3 * g.M;
        if (cudaMalloc(&sv[i].R, n * es) != cudaSuccess || cudaMalloc(&sv[i].com, (size_t)g.C * 24) != cudaSuccess ||
            cudaMalloc(&sv[i].step, (size_t)g.C * 8) != cudaSuccess) {
            release();
            return fail(SFP_ENOMEM, "autotune: no memory for the state copy");
        }
        CUDA_TRY(cudaMemcpyAsync(sv[i].R, g.R, n * es, cudaMemcpyDeviceToDevice, b->stream));
        CUDA_TRY(cudaMemcpyAsync(sv[i].com, g.com, (size_t)g.C * 24, cudaMemcpyDeviceToDevice, b->stream));
        CUDA_TRY(cudaMemcpyAsync(sv[i].step, g.step, (size_t)g.C * 8, cudaMemcpyDeviceToDevice, b->stream));
    }
    auto restore = [&]() -> int {
        for (size_t i = 0; i < G; ++i) {
            const Group& g = b->groups[i];
            const size_t n = (size_t)g.C * 3 * g.M;
            CUDA_TRY(cudaMemcpyAsync(g.R, sv[i].R, n * es, cudaMemcpyDeviceToDevice, b->stream));
            CUDA_TRY(cudaMemcpyAsync(g.com, sv[i].com, (size_t)g.C * 24, cudaMemcpyDeviceToDevice, b->stream));
            CUDA_TRY(cudaMemcpyAsync(g.step, sv[i].step, (size_t)g.C * 8, cudaMemcpyDeviceToDevice, b->stream));
        }
        return SFP_OK;
    };
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // time `fn` (warm-up, then one timed call) on the batch stream, restoring the state after each
    auto timed = [&](auto&& fn, double* ms) -> int {
        int rc = fn();
        if (!rc) rc = restore();
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(e0, b->stream));
        if ((rc = fn())) return rc;
        CUDA_TRY(cudaEventRecord(e1, b->stream));
        CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        *ms = t;
        return restore();
    };
    const bool was_graph = b->use_graph;
    drop_graph(b);
    b->use_graph = false;
    int rc = SFP_OK;
    // 1. each fused group alone, for a few chains-per-tile candidates
    std::vector<std::vector<std::pair<int, double>>> cand(fg.size());
    for (size_t k = 0; k < fg.size() && !rc; ++k) {
        Group& g = b->groups[fg[k]];
        std::vector<int> cs;
        const int units = sms / sfp::fused_ctas_per_tile(g.fused);   // tiles that fit one wave
        for (double f : {1.0, 0.75, 0.5, 1.0 / 3.0, 0.25}) {
            const int target = std::max(1, (int)(f * units));
            cs.push_back(std::min(40, ((g.C + target - 1) / target + 3) / 4 * 4));
        }
        cs.push_back(40);
        std::sort(cs.begin(), cs.end());
        cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
        for (int c : cs) {
            if ((rc = sfp::fused_set_tile(g.fused, c))) break;
            double ms = 0.0;
            b->cur = b->stream;
            rc = timed([&]() { return step_group_fused(b, g, trial_steps); }, &ms);
            if (rc) break;
            cand[k].push_back({c, ms});
        }
    }
    // 2. combinations: estimated concurrent makespan max(max t, sum t * CTAs / SMs),
    //    then the best estimate and the best-alone choice are measured together
    std::vector<int> best_alone(fg.size()), best_est(fg.size());
    if (!rc) {
        for (size_t k = 0; k < fg.size(); ++k)
            best_alone[k] = std::min_element(cand[k].begin(), cand[k].end(),
                                             [](auto& x, auto& y) { return x.second < y.second; })->first;
        double best = 1e300;
        std::vector<size_t> idx(fg.size(), 0);
        for (;;) {
            double mx = 0.0, share = 0.0;
            for (size_t k = 0; k < fg.size(); ++k) {
                const auto& cnd = cand[k][idx[k]];
                const Group& g = b->groups[fg[k]];
                mx = std::max(mx, cnd.second);
                share += cnd.second * (double)((g.C + cnd.first - 1) / cnd.first) *
                         sfp::fused_ctas_per_tile(g.fused) / sms;
            }
            const double est = std::max(mx, share);
            if (est < best) {
                best = est;
                for (size_t k = 0; k < fg.size(); ++k) best_est[k] = cand[k][idx[k]].first;
            }
            size_t k = 0;
            while (k < fg.size() && ++idx[k] == cand[k].size()) idx[k++] = 0;
            if (k == fg.size()) break;
        }
        double t_est = 0.0, t_alone = 0.0;
        auto set_all = [&](const std::vector<int>& v) -> int {
            for (size_t k = 0; k < fg.size(); ++k) {
                const int r = sfp::fused_set_tile(b->groups[fg[k]].fused, v[k]);
                if (r) return r;
            }
            return SFP_OK;
        };
        auto whole = [&]() { return issue_chunk(b, trial_steps, b->stream); };
        if (!(rc = set_all(best_est))) rc = timed(whole, &t_est);
        if (!rc && best_alone != best_est && !(rc = set_all(best_alone))) rc = timed(whole, &t_alone);
        if (!rc && best_alone != best_est && t_est <= t_alone) rc = set_all(best_est);
    }
    b->cur = b->stream;
    b->use_graph = was_graph;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rr = restore();
    cudaStreamSynchronize(b->stream);
    release();
    if (rc) return rc;
    if (rr) return rr;
    if (chains_per_tile)
        for (size_t i = 0; i < G; ++i) chains_per_tile[i] = b->groups[i].fused ? sfp::fused_tile(b->groups[i].fused) : 0;
    return SFP_OK;
}

int sfp_set_integrator(sfp_batch* b, int32_t integrator)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (integrator != SFP_INTEGRATOR_MODES && integrator != SFP_INTEGRATOR_EULER)
        return fail(SFP_EINVAL, "unknown integrator %d", integrator);
    for (const auto& g : b->groups)
        if (g.limited) return fail(SFP_ENOTSUP, "serving pools step in mode space only");
    if (b->integrator != integrator) drop_graph(b);
    b->integrator = integrator;
    return SFP_OK;
}

int sfp_set_sampling(sfp_batch* b, int32_t every_steps)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    if (every_steps < 0) return fail(SFP_EINVAL, "every_steps < 0");
    if (every_steps == 0) {
        b->sample_every = 0;
        return SFP_OK;
    }
    int rc;
    for (auto& g : b->groups) {
        const int M = g.M, N = M - 1;
        if (!g.obs_tab) {
            if ((rc = dalloc_t(b, &g.obs_tab, (size_t)3 * M * 8)) ||
                (rc = dalloc_t(b, &g.acc_shape, (size_t)g.C * 4 * 8)) ||
                (rc = dalloc_t(b, &g.acc_pow, (size_t)g.C * 3 * M * 8)) ||
                (rc = dalloc_t(b, &g.msd_snap, (size_t)g.C * sfp::kMaxLags * 3 * 8)) ||
                (rc = dalloc_t(b, &g.msd_acc, (size_t)g.C * sfp::kMaxLags * 2 * 8)) ||
                (rc = dalloc_t(b, &g.mid_snap, (size_t)g.C * sfp::kMaxLags * 3 * 8)) ||
                (rc = dalloc_t(b, &g.mid_acc, (size_t)g.C * sfp::kMaxLags * 2 * 8)) ||
                (rc = dalloc_t(b, &g.e2e_snap, (size_t)g.C * sfp::kMaxLags * 3 * 8)) ||
                (rc = dalloc_t(b, &g.e2e_acc, (size_t)g.C * sfp::kMaxLags * 2 * 8)) ||
                (rc = dalloc_t(b, &g.bond_snap, (size_t)g.C * sfp::kMaxLags * 3 * 8)) ||
                (rc = dalloc_t(b, &g.bond_acc, (size_t)g.C * sfp::kMaxLags * 2 * 8)))
                return rc;
            // coefficient rows of L = r_N - r_0, u_m = r_m - r_{m-1} (m = ceil(N/2)) and
            // r_m' - r_cm (m' = floor(N/2)) in terms of R_p (Eq. c1); p = 0 drops out of all three
            std::vector<double> t((size_t)3 * M, 0.0);
            const int mb = (N + 1) / 2, mm = N / 2;
            const auto& phi = g.tab.phi;
            for (int p = 1; p < M; ++p) {
                t[p] = phi[(size_t)N * M + p] - phi[p];
                t[M + p] = phi[(size_t)mb * M + p] - phi[(size_t)(mb - 1) * M + p];
                t[2 * M + p] = phi[(size_t)mm * M + p];
            }
            CUDA_TRY(cudaMemcpyAsync(g.obs_tab, t.data(), t.size() * 8, cudaMemcpyHostToDevice, b->stream));
            CUDA_TRY(cudaStreamSynchronize(b->stream));
        }
        CUDA_TRY(cudaMemsetAsync(g.acc_shape, 0, (size_t)g.C * 4 * 8, b->stream));
        CUDA_TRY(cudaMemsetAsync(g.acc_pow, 0, (size_t)g.C * 3 * M * 8, b->stream));
        CUDA_TRY(cudaMemsetAsync(g.msd_snap, 0, (size_t)g.C * sfp::kMaxLags * 3 * 8, b->stream));
        CUDA_TRY(cudaMemsetAsync(g.msd_acc, 0, (size_t)g.C * sfp::kMaxLags * 2 * 8, b->stream));
        for (double* x : {g.mid_snap, g.e2e_snap, g.bond_snap})
            CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)g.C * sfp::kMaxLags * 3 * 8, b->stream));
        for (double* x : {g.mid_acc, g.e2e_acc, g.bond_acc})
            CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)g.C * sfp::kMaxLags * 2 * 8, b->stream));
    }
    b->lags = b->lags_next;
    b->sampled = true;
    b->sample_every = every_steps;
    b->n_samples = 0;
    return sample_all(b);
}

int sfp_set_msd_lags(sfp_batch* b, int32_t n_lags, const int32_t* lags)
{
    if (!b || !lags) return fail(SFP_EINVAL, "NULL argument");
    if (n_lags < 1 || n_lags > sfp::kMaxLags) return fail(SFP_EINVAL, "n_lags must be 1..%d", sfp::kMaxLags);
    sfp::SampleLags L{};
    L.n = n_lags;
    for (int i = 0; i < n_lags; ++i) {
        if (lags[i] < 1) return fail(SFP_EINVAL, "lag %d is %d; lags are >= 1 sampling intervals", i, lags[i]);
        L.v[i] = lags[i];
    }
    b->lags_next = L;
    return SFP_OK;
}

int sfp_philox_words(uint32_t seed, uint32_t job, int64_t step, uint32_t tag, int32_t count,
                     uint32_t* host_out)
{
    if (!host_out || count <= 0) return fail(SFP_EINVAL, "need count > 0 and an output buffer");
    uint32_t* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, (size_t)count * 16));
    sfp::k_philox_words<<<nblk(count, 128), 128>>>(seed, job, step, tag, count, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, (size_t)count * 16, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(SFP_ECUDA, "philox words: %s", cudaGetErrorString(e));
    return SFP_OK;
}

int sfp_step_noalloc(const sfp_params* params, const sfp_chain_desc* chain, int32_t n_chains,
                     uint64_t seed, int64_t step0, float* modes_dev, double* com_dev, int64_t n_steps,
                     void* cuda_stream)
{
    if (!chain || !modes_dev || !com_dev) return fail(SFP_EINVAL, "NULL argument");
    if (n_chains <= 0 || n_steps < 0 || step0 < 0) return fail(SFP_EINVAL, "need n_chains > 0, n_steps >= 0, step0 >= 0");
    if (seed >> 32) return fail(SFP_EINVAL, "seed must be < 2^32");
    if (chain->reserved != 0) return fail(SFP_EINVAL, "reserved must be 0");
    if ((chain->job_id >> 32) || chain->job_id + (uint64_t)n_chains - 1 >= (1ull << 32))
        return fail(SFP_EINVAL, "job_id + n_chains - 1 must be < 2^32");
    if (chain->n_beads < 3 || chain->n_beads > 4096) return fail(SFP_EINVAL, "n_beads %d outside 3..4096", chain->n_beads);
    Derived dv;
    int rc = derive(params, &dv);
    if (rc) return rc;
    const double dtau = chain->dtau > 0.0 ? chain->dtau : chain->dt_ps / dv.c_ps;
    if (!(dtau > 0.0) || !std::isfinite(dtau)) return fail(SFP_EINVAL, "step must be > 0");
    if (!std::isfinite(chain->shear_rate_per_s)) return fail(SFP_EINVAL, "shear rate not finite");
    const int M = chain->n_beads, C = n_chains;
    const size_t fM = (size_t)M * sizeof(float), n = (size_t)C * 3 * M;
    // carve the array: chi | chiT | phiT | dm h w g | u | v z | DeltaH Z | step | job | shear | flag
    size_t off = 0;
    auto take = [&off](size_t bytes) { const size_t o = off; off += align256(bytes); return o; };
    const size_t o_chi = take(fM * M), o_chiT = take(fM * M), o_phiT = take(fM * M), o_dm = take(fM),
                 o_h = take(fM), o_w = take(fM),
                 o_g = take(fM), o_r = take(n * 4), o_fz = take(2 * n * 4), o_yz = take(2 * n * 4),
                 o_step = take((size_t)C * 8), o_job = take((size_t)C * 4), o_sh = take((size_t)C * 8),
                 o_bad = take(sizeof(int));
    if (off > (size_t)SFP_NOALLOC_SCRATCH_BYTES)
        return fail(SFP_EINVAL, "%d chains x %d beads need %zu bytes of scratch; the static array holds %u",
                    C, M, off, (unsigned)SFP_NOALLOC_SCRATCH_BYTES);
    unsigned char* base = nullptr;
    if ((rc = noalloc_scratch(&base))) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    float* chi = (float*)(base + o_chi);
    float* chiT = (float*)(base + o_chiT);
    float* phiT = (float*)(base + o_phiT);
    float *dm = (float*)(base + o_dm), *h = (float*)(base + o_h), *w = (float*)(base + o_w), *g = (float*)(base + o_g);
    float* r = (float*)(base + o_r);
    float* fz = (float*)(base + o_fz);
    float* yz = (float*)(base + o_yz);
    int64_t* step = (int64_t*)(base + o_step);
    uint32_t* job = (uint32_t*)(base + o_job);
    double* shear = (double*)(base + o_sh);
    k_noalloc_tables<<<nblk((int64_t)M * M, 256), 256, 0, st>>>(chi, chiT, phiT, dm, h, w, g, M, dv.Tstar, dv.nu,
                                                                 dtau);
    k_noalloc_prep<<<nblk(C, 128), 128, 0, st>>>(modes_dev, step, job, shear, (int*)(base + o_bad), C, M, step0,
                                                  (uint32_t)chain->job_id, chain->shear_rate_per_s * dv.c_ps * 1e-12);
    CUDA_TRY(cudaGetLastError());
    const float c12 = (float)(1.0 - 2.0 * dv.nu);
    const double w0 = std::sqrt(2.0 * dv.Tstar * dtau);
    int* bad = (int*)(base + o_bad);   // written by the update kernel, not reported here
    for (int64_t s = 0; s < n_steps; ++s) {
        CUDA_TRY(gemm_on<float>(st, modes_dev, chi, r, 3 * C, M, M));
        CUDA_TRY(launch_force<float>(st, r, fz, C, M, c12));
        CUDA_TRY(launch_noise<float>(st, fz + n, C, M, (uint32_t)seed, job, step));
        CUDA_TRY(gemm_on<float>(st, fz, chiT, yz, 3 * C, M, M));
        CUDA_TRY(gemm_on<float>(st, fz + n, phiT, yz + n, 3 * C, M, M));
        CUDA_TRY(launch_mode_update<float>(st, modes_dev, yz, yz + n, com_dev, step, dm, h, w, g, shear, C, M, w0,
                                           dtau, bad, nullptr));
    }
    return SFP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Slot access for the serving loop (sfp_server.cu); single-group batches.
// ---------------------------------------------------------------------------
namespace {
constexpr int kGather = 256;   // slots read back per launch

int slot_buffers(sfp_batch* b, Group& g)
{
    if (g.slot_idx) return SFP_OK;
    int rc;
    const int N = g.M - 1;
    if ((rc = dalloc_t(b, &g.rod, (size_t)3 * N * 8)) || (rc = dalloc_t(b, &g.slot_idx, (size_t)g.C * 4)) ||
        (rc = dalloc_t(b, &g.read_idx, (size_t)kGather * 4)) ||
        (rc = dalloc_t(b, &g.slot_job, (size_t)g.C * 4)) || (rc = dalloc_t(b, &g.slot_stop, (size_t)g.C * 8)) ||
        (rc = dalloc_t(b, &g.slot_shear, (size_t)g.C * 8)) ||
        (rc = dalloc_t(b, &g.gather, (size_t)kGather * (3 * g.M + 4) * 8)))
        return rc;
    std::vector<double> l0, Ld, Lo;
    rod_tables(g.M, b->dv.nu, &l0, &Ld, &Lo);
    std::vector<double> all;
    all.insert(all.end(), l0.begin(), l0.end());
    all.insert(all.end(), Ld.begin(), Ld.end());
    all.insert(all.end(), Lo.begin(), Lo.end());
    CUDA_TRY(cudaMemcpyAsync(g.rod, all.data(), all.size() * 8, cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    return SFP_OK;
}
}  // namespace

int sfp::internal_idle_all(sfp_batch* b)
{
    if (!b || b->groups.size() != 1) return fail(SFP_EINVAL, "serving pools hold one length group");
    Group& g = b->groups[0];
    const int rc = slot_buffers(b, g);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(g.stop, 0, (size_t)g.C * 8, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    g.limited = true;
    return SFP_OK;
}

int sfp::internal_slots_start(sfp_batch* b, const int32_t* slots, const uint32_t* jobs, const int64_t* stops,
                              const double* shear_per_s, int32_t n)
{
    if (!b || b->groups.size() != 1) return fail(SFP_EINVAL, "serving pools hold one length group");
    if (n <= 0) return SFP_OK;
    Group& g = b->groups[0];
    if (n > g.C) return fail(SFP_EINVAL, "more slots than the pool holds");
    for (int i = 0; i < n; ++i)
        if (slots[i] < 0 || slots[i] >= g.C) return fail(SFP_EINVAL, "slot %d out of range", slots[i]);
    int rc = slot_buffers(b, g);
    if (rc) return rc;
    std::vector<double> sh(n);
    for (int i = 0; i < n; ++i) sh[i] = shear_per_s[i] * b->dv.c_ps * 1e-12;   // 1/s -> 1/tau
    CUDA_TRY(cudaMemcpyAsync(g.slot_idx, slots, (size_t)n * 4, cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaMemcpyAsync(g.slot_job, jobs, (size_t)n * 4, cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaMemcpyAsync(g.slot_stop, stops, (size_t)n * 8, cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaMemcpyAsync(g.slot_shear, sh.data(), (size_t)n * 8, cudaMemcpyHostToDevice, b->stream));
    const int N = g.M - 1;
    const size_t smem = (size_t)4 * g.M * 8;
    if (b->precision == SFP_FP64) {
        if (smem > 48 * 1024)
            CUDA_TRY(cudaFuncSetAttribute(sfp::k_init_slots<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sfp::k_init_slots<double><<<n, 128, smem, b->stream>>>((double*)g.R, g.com, g.step, g.stop, g.job, g.shear,
            g.slot_idx, g.slot_job, g.slot_stop, g.slot_shear, g.phi_d, g.rod, g.rod + N, g.rod + 2 * N,
            g.M, b->dv.Tstar, b->dv.nu, b->seed);
    } else {
        if (smem > 48 * 1024)
            CUDA_TRY(cudaFuncSetAttribute(sfp::k_init_slots<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sfp::k_init_slots<float><<<n, 128, smem, b->stream>>>((float*)g.R, g.com, g.step, g.stop, g.job, g.shear,
            g.slot_idx, g.slot_job, g.slot_stop, g.slot_shear, g.phi_d, g.rod, g.rod + N, g.rod + 2 * N,
            g.M, b->dv.Tstar, b->dv.nu, b->seed);
    }
    CUDA_TRY(cudaGetLastError());
    g.limited = true;
    b->probed = false;
    return SFP_OK;
}

int sfp::internal_slots_read(sfp_batch* b, const int32_t* slots, int32_t n, double* modes, double* com_nm,
                             int64_t* steps, cudaStream_t stream, cudaEvent_t after)
{
    if (!b || b->groups.size() != 1) return fail(SFP_EINVAL, "serving pools hold one length group");
    Group& g = b->groups[0];
    int rc = slot_buffers(b, g);
    if (rc) return rc;
    const int M = g.M;
    cudaStream_t st_r = stream ? stream : b->stream;
    if (after) CUDA_TRY(cudaStreamWaitEvent(st_r, after, 0));
    for (int i0 = 0; i0 < n; i0 += kGather) {
        const int k = std::min(kGather, n - i0);
        for (int i = 0; i < k; ++i)
            if (slots[i0 + i] < 0 || slots[i0 + i] >= g.C) return fail(SFP_EINVAL, "slot out of range");
        double* out = g.gather;
        double* cm = out + (size_t)kGather * 3 * M;
        int64_t* st = (int64_t*)(cm + (size_t)kGather * 3);
        CUDA_TRY(cudaMemcpyAsync(g.read_idx, slots + i0, (size_t)k * 4, cudaMemcpyHostToDevice, st_r));
        if (b->precision == SFP_FP64)
            sfp::k_gather_slots<double><<<k, 128, 0, st_r>>>((const double*)g.R, g.com, g.step, g.read_idx, k, M, out, cm, st);
        else
            sfp::k_gather_slots<float><<<k, 128, 0, st_r>>>((const float*)g.R, g.com, g.step, g.read_idx, k, M, out, cm, st);
        CUDA_TRY(cudaGetLastError());
        if (modes) CUDA_TRY(cudaMemcpyAsync(modes + (size_t)i0 * 3 * M, out, (size_t)k * 3 * M * 8, cudaMemcpyDeviceToHost, st_r));
        std::vector<double> c3((size_t)k * 3);
        CUDA_TRY(cudaMemcpyAsync(c3.data(), cm, c3.size() * 8, cudaMemcpyDeviceToHost, st_r));
        if (steps) CUDA_TRY(cudaMemcpyAsync(steps + i0, st, (size_t)k * 8, cudaMemcpyDeviceToHost, st_r));
        CUDA_TRY(cudaStreamSynchronize(st_r));
        if (com_nm)
            for (size_t i = 0; i < c3.size(); ++i) com_nm[(size_t)i0 * 3 + i] = c3[i] * b->dv.d_nm;
    }
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, b->bad, sizeof(int), cudaMemcpyDeviceToHost, st_r));
    CUDA_TRY(cudaStreamSynchronize(st_r));
    if (bad & 4) return fail(SFP_ECUDA, "a 512-bead fused step ran without its two-CTA cluster");
    if (bad & 2) return fail(SFP_ETIMEDOUT, "a tensor-core pipeline wait timed out");
    if (bad & 1) return fail(SFP_ENONFINITE, "a chain's state became non-finite");
    return SFP_OK;
}

int sfp::internal_set_active(sfp_batch* b, int64_t n)
{
    if (!b) return fail(SFP_EINVAL, "batch is NULL");
    b->active_limit = n;
    return SFP_OK;
}

int sfp::internal_shape(const sfp_batch* b, int32_t* M, double* dtau, int32_t* C, size_t* bytes)
{
    if (!b || b->groups.empty()) return fail(SFP_EINVAL, "empty batch");
    if (M) *M = b->groups[0].M;
    if (dtau) *dtau = b->groups[0].dtau;
    if (C) *C = b->groups[0].C;
    if (bytes) *bytes = b->held;
    return SFP_OK;
}
