/*
 * sfp_oracle.c -- plain FP64 CPU oracle for the mode-space Langevin step of
 * the extensible bead-spring model of Panja, Barkema and van Leeuwen,
 * "Efficient simulation of semiflexible polymers" (arXiv:1411.3487).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything is in the paper's scaled units (Sec. 3, Eqs. b3-b5): lengths in
 * units of d, time in units of xi/lambda.  Beads n = 0..N, bonds n = 1..N,
 * modes p = 0..N, M = N+1.  Arrays of vectors are stored axis-major:
 * x[alpha*M + n] for alpha = 0,1,2.
 *
 * Readings of the paper taken here, where a passage is ambiguous or garbled:
 *   - Eq. c8 is printed with sqrt(2/(N+1)) for every p and "p = 0..N-1";
 *     the transform is square and orthonormal only with p = 0..N and
 *     phi_{n,0} = 1/sqrt(N+1) (Eq. c2).
 *   - chi_{n,p} is defined as phi_{n,p} - phi_{n-1,p} (Eq. e3, first form).
 *   - H_p = +dL_c/dR_p (Eq. e1), which follows from H' = H* - L_c (Eq. c6).
 *   - Eq. f0 carries zeta^t_p; Eqs. d5/e10 carry zeta_p (Eq. e9), used here.
 *   - p = 0 (centre of mass): zeta_0 = 0, DeltaH_0 = 0, so h_0 = 0 and the
 *     noise amplitude is the zeta -> 0 limit of Eq. d6, sqrt(2 T* dtau).
 *   - Noise is drawn per bead and projected (Eq. c4): Z_p = sum_n phi z_n.
 *   - Shear (Eq. btum) in mode space: dR^x_p/dtau gains gamma R^y_p; it is
 *     integrated with R^y held at its start-of-step value.
 *
 * Also here: the Metropolis Monte Carlo sampler in mode amplitudes that the
 * paper uses as its equilibrium benchmark (Sec. 5A), orc_mc_sweeps.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
 * from its published definition.  key = (seed, job_id); counter =
 * (step_lo, step_hi, index, tag).  Uniforms use the top 23 bits,
 * u = (floor(x / 2^9) + 1/2) / 2^23, so they are exact in FP32 as well.
 * Box-Muller on the word pairs (x0,x1) and (x2,x3) gives four normals per
 * call, all used: the normal of bead n, axis alpha is number k = 3n + alpha
 * of the step, value k mod 4 of the call with index k / 4.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                              */
/* ------------------------------------------------------------------------ */

static void philox_round(uint32_t x[4], const uint32_t k[2])
{
    /* One Philox S-box round: two 32x32->64 multiplies, then a Feistel-like
     * mix of the high halves with the other two words and the round key. */
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ x[1] ^ k[0];
    const uint32_t y1 = lo1;
    const uint32_t y2 = hi0 ^ x[3] ^ k[1];
    const uint32_t y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }  /* Weyl key schedule */
        philox_round(x, k);
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

double orc_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);   /* 2^-23 */
}

/* Four standard normals from Philox call `call` of one chain: Box-Muller on
 * the word pairs (0,1) and (2,3), both values of each pair used. */
static void normals4(uint32_t seed, uint32_t job, int64_t step, uint32_t call,
                     uint32_t tag, double n4[4])
{
    const uint32_t ctr[4] = {(uint32_t)((uint64_t)step & 0xffffffffu),
                             (uint32_t)((uint64_t)step >> 32), call, tag};
    const uint32_t key[2] = {seed, job};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    const double ra = sqrt(-2.0 * log(orc_u01(x[0])));
    const double ta = 2.0 * ORC_PI * orc_u01(x[1]);
    const double rb = sqrt(-2.0 * log(orc_u01(x[2])));
    const double tb = 2.0 * ORC_PI * orc_u01(x[3]);
    n4[0] = ra * cos(ta);
    n4[1] = ra * sin(ta);
    n4[2] = rb * cos(tb);
    n4[3] = rb * sin(tb);
}

/* z[alpha*M + n] ~ N(0,1): the per-bead thermal noise of step `step`.  The
 * normal of bead n, axis alpha has index k = 3n + alpha and is value k mod 4
 * of Philox call k / 4, so the 3M normals of a step take ceil(3M/4) calls. */
void orc_bead_normals(uint32_t seed, uint32_t job, int64_t step, uint32_t tag,
                      int M, double *z)
{
    const int K = 3 * M;
    for (int call = 0; 4 * call < K; ++call) {
        double g[4];
        normals4(seed, job, step, (uint32_t)call, tag, g);
        for (int e = 0; e < 4 && 4 * call + e < K; ++e) {
            const int k = 4 * call + e;
            z[(k % 3) * M + k / 3] = g[e];
        }
    }
}

/* Z[alpha*M + p] ~ N(0,1): noise drawn per mode instead of per bead (the
 * mode-keyed variant).  Projecting iid normals through the orthonormal phi
 * (Eq. c4, Z = phi^T z) gives iid normals again, so drawing Z directly has the
 * same distribution.  Normal k = 3p + alpha is value k mod 4 of Philox call
 * k / 4 with tag 2 (the bead noise has tag 0, the start sampler tag 1). */
void orc_mode_normals(uint32_t seed, uint32_t job, int64_t step, int M, double *Z)
{
    orc_bead_normals(seed, job, step, 2u, M, Z);
}

/* ------------------------------------------------------------------------ */
/* Model tables (Secs. 3A, 4, 4A, 4B)                                        */
/* ------------------------------------------------------------------------ */

typedef struct orc_model {
    int M;                 /* beads = modes = N+1 */
    double Tstar, nu, dtau;
    double *phi;           /* phi[n*M + p], Eq. c8 (orthonormal at p = 0) */
    double *chi;           /* chi[(n-1)*M + p] for bonds n = 1..N, Eq. e3 */
    double *zl;            /* zeta^l_p, Eq. c9 */
    double *zeta;          /* zeta_p, Eq. e9 */
    double *decay;         /* exp(-zeta_p dtau), Eq. d3 */
    double *h;             /* DeltaH integration weight, Eq. f2 */
    double *w;             /* noise amplitude, Eq. d6 */
    double *g;             /* shear weight: int_0^dtau exp(-zeta_p s) ds */
} orc_model;

void orc_model_free(orc_model *m)
{
    if (!m) return;
    free(m->phi); free(m->chi); free(m->zl); free(m->zeta);
    free(m->decay); free(m->h); free(m->w); free(m->g);
    free(m);
}

orc_model *orc_model_new(int M, double Tstar, double nu, double dtau)
{
    if (M < 2 || !(nu > 0.0 && nu < 0.5) || !(Tstar >= 0.0) || !(dtau > 0.0)) return NULL;
    orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
    if (!m) return NULL;
    const int N = M - 1;
    m->M = M; m->Tstar = Tstar; m->nu = nu; m->dtau = dtau;
    m->phi = (double *)malloc(sizeof(double) * (size_t)M * M);
    m->chi = (double *)malloc(sizeof(double) * (size_t)N * M);
    m->zl = (double *)malloc(sizeof(double) * M);
    m->zeta = (double *)malloc(sizeof(double) * M);
    m->decay = (double *)malloc(sizeof(double) * M);
    m->h = (double *)malloc(sizeof(double) * M);
    m->w = (double *)malloc(sizeof(double) * M);
    m->g = (double *)malloc(sizeof(double) * M);
    if (!m->phi || !m->chi || !m->zl || !m->zeta || !m->decay || !m->h || !m->w || !m->g) {
        orc_model_free(m);
        return NULL;
    }
    /* Eq. c8: phi_{n,p} = sqrt(2/(N+1)) cos(p (n+1/2) pi / (N+1)), p >= 1;
     * phi_{n,0} = 1/sqrt(N+1) so that Eq. c2 holds. */
    for (int n = 0; n < M; ++n)
        for (int p = 0; p < M; ++p)
            m->phi[(size_t)n * M + p] = (p == 0)
                ? 1.0 / sqrt((double)M)
                : sqrt(2.0 / M) * cos(p * (n + 0.5) * ORC_PI / M);
    /* Eq. e3: chi_{n,p} = phi_{n,p} - phi_{n-1,p}, bonds n = 1..N. */
    for (int n = 1; n <= N; ++n)
        for (int p = 0; p < M; ++p)
            m->chi[(size_t)(n - 1) * M + p] =
                m->phi[(size_t)n * M + p] - m->phi[(size_t)(n - 1) * M + p];
    for (int p = 0; p < M; ++p) {
        const double th = p * ORC_PI / M;
        /* Eq. c9 */
        m->zl[p] = 2.0 * (1.0 - cos(th)) * (1.0 - 2.0 * nu * cos(th));
        /* Eq. e9 */
        const double s = 2.0 * sin(th / 2.0);
        m->zeta[p] = m->zl[p] - (1.0 - 2.0 * nu) * s * s;
        if (p == 0) {
            m->decay[p] = 1.0;
            m->h[p] = 0.0;
            m->w[p] = sqrt(2.0 * Tstar * dtau);
            m->g[p] = dtau;
            continue;
        }
        /* Eq. d3 */
        m->decay[p] = exp(-m->zeta[p] * dtau);
        /* Eq. f2 */
        m->h[p] = (exp(-m->zeta[p] * dtau) - exp(-m->zl[p] * dtau)) / (m->zl[p] - m->zeta[p]);
        /* Eq. d6 */
        m->w[p] = sqrt(Tstar * (1.0 - exp(-2.0 * m->zeta[p] * dtau)) / m->zeta[p]);
        /* shear: R^y held over the step, integrated against the OU kernel of Eq. d5 */
        m->g[p] = (1.0 - exp(-m->zeta[p] * dtau)) / m->zeta[p];
    }
    return m;
}

/* Copy the tables out (any pointer may be NULL). */
void orc_model_tables(const orc_model *m, double *phi, double *chi, double *zl,
                      double *zeta, double *decay, double *h, double *w, double *g)
{
    const size_t M = (size_t)m->M;
    if (phi) memcpy(phi, m->phi, sizeof(double) * M * M);
    if (chi) memcpy(chi, m->chi, sizeof(double) * (M - 1) * M);
    if (zl) memcpy(zl, m->zl, sizeof(double) * M);
    if (zeta) memcpy(zeta, m->zeta, sizeof(double) * M);
    if (decay) memcpy(decay, m->decay, sizeof(double) * M);
    if (h) memcpy(h, m->h, sizeof(double) * M);
    if (w) memcpy(w, m->w, sizeof(double) * M);
    if (g) memcpy(g, m->g, sizeof(double) * M);
}

/* ------------------------------------------------------------------------ */
/* Single-chain primitives                                                    */
/* ------------------------------------------------------------------------ */

/* Eq. c1, second line: r_n = sum_p phi_{n,p} R_p (all p, centre of mass included). */
void orc_modes_to_beads(const orc_model *m, const double *R, double *r)
{
    const int M = m->M;
    for (int a = 0; a < 3; ++a)
        for (int n = 0; n < M; ++n) {
            double s = 0.0;
            for (int p = 0; p < M; ++p) s += m->phi[(size_t)n * M + p] * R[a * M + p];
            r[a * M + n] = s;
        }
}

/* Eq. c1, first line: R_p = sum_n r_n phi_{n,p}. */
void orc_beads_to_modes(const orc_model *m, const double *r, double *R)
{
    const int M = m->M;
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p < M; ++p) {
            double s = 0.0;
            for (int n = 0; n < M; ++n) s += r[a * M + n] * m->phi[(size_t)n * M + p];
            R[a * M + p] = s;
        }
}

/* Eq. e11: DeltaH_p = sum_{n=1}^N chi_{n,p} u_n [1/|u_n| - (1 - 2 nu)],
 * with the bond vectors u_n = r_n - r_{n-1} taken from bead positions r. */
void orc_delta_H(const orc_model *m, const double *r, double *dH)
{
    const int M = m->M, N = M - 1;
    const double c = 1.0 - 2.0 * m->nu;
    double *v = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    for (int n = 1; n <= N; ++n) {
        const double ux = r[n] - r[n - 1];
        const double uy = r[M + n] - r[M + n - 1];
        const double uz = r[2 * M + n] - r[2 * M + n - 1];
        const double len = sqrt(ux * ux + uy * uy + uz * uz);
        const double s = 1.0 / len - c;
        v[n] = ux * s; v[M + n] = uy * s; v[2 * M + n] = uz * s;
    }
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p < M; ++p) {
            double s = 0.0;
            for (int n = 1; n <= N; ++n) s += m->chi[(size_t)(n - 1) * M + p] * v[a * M + n];
            dH[a * M + p] = s;
        }
    free(v);
}

/* Scaled energy H' = T* H/kT of Eq. a2: 1/2 sum (|u_n|-1)^2 - nu sum u_n.u_{n+1}. */
double orc_energy(const orc_model *m, const double *r)
{
    const int M = m->M, N = M - 1;
    double e = 0.0, px = 0, py = 0, pz = 0;
    for (int n = 1; n <= N; ++n) {
        const double ux = r[n] - r[n - 1];
        const double uy = r[M + n] - r[M + n - 1];
        const double uz = r[2 * M + n] - r[2 * M + n - 1];
        const double len = sqrt(ux * ux + uy * uy + uz * uz);
        e += 0.5 * (len - 1.0) * (len - 1.0);
        if (n >= 2) e -= m->nu * (ux * px + uy * py + uz * pz);
        px = ux; py = uy; pz = uz;
    }
    return e;
}

/* Bead force F_n = -dH'/dr_n for the default bead-position scheme (Eq. b3):
 * with e_n = dH'/du_n = (|u_n|-1) u_n/|u_n| - nu (u_{n-1} + u_{n+1}) and
 * u_0 = u_{N+1} = 0, e_0 = e_{N+1} = 0, F_n = e_{n+1} - e_n. */
void orc_full_force(const orc_model *m, const double *r, double *F)
{
    const int M = m->M, N = M - 1;
    double *u = (double *)calloc(3 * (size_t)(M + 1), sizeof(double));  /* u[a*(M+1)+n], n=0..N+1 */
    double *e = (double *)calloc(3 * (size_t)(M + 1), sizeof(double));
    const int S = M + 1;
    for (int a = 0; a < 3; ++a)
        for (int n = 1; n <= N; ++n) u[a * S + n] = r[a * M + n] - r[a * M + n - 1];
    for (int n = 1; n <= N; ++n) {
        const double len = sqrt(u[n] * u[n] + u[S + n] * u[S + n] + u[2 * S + n] * u[2 * S + n]);
        for (int a = 0; a < 3; ++a)
            e[a * S + n] = (len - 1.0) * u[a * S + n] / len
                         - m->nu * (u[a * S + n - 1] + u[a * S + n + 1]);
    }
    for (int a = 0; a < 3; ++a)
        for (int n = 0; n <= N; ++n) F[a * M + n] = e[a * S + n + 1] - e[a * S + n];
    free(u); free(e);
}

/* One mode-space step (Sec. 4) of one chain with the bead noise z given:
 *   r = phi R (Eq. c1); DeltaH (Eq. e11); Z = phi^T z (Eq. c4);
 *   R_p <- exp(-zeta_p dtau) R_p + h_p DeltaH_p + w_p Z_p   (Eqs. d3, d6, f2)
 *   R^x_p += shear * g_p * R^y_p(start of step)               (Eq. btum)
 * coupling = 0 drops DeltaH (the pure Ornstein-Uhlenbeck case of Eq. d3). */
void orc_mode_step_Zm(const orc_model *m, const double *Z, double shear, int coupling, double *R);

void orc_mode_step_z(const orc_model *m, const double *z, double shear, int coupling, double *R)
{
    const int M = m->M;
    double *Z = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    orc_beads_to_modes(m, z, Z);
    orc_mode_step_Zm(m, Z, shear, coupling, R);
    free(Z);
}

/* The same step with the mode noise Z given (Z = phi^T z for bead noise z,
 * or drawn per mode by orc_mode_normals). */
void orc_mode_step_Zm(const orc_model *m, const double *Z, double shear, int coupling, double *R)
{
    const int M = m->M;
    double *r = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    double *dH = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    orc_modes_to_beads(m, R, r);
    if (coupling) orc_delta_H(m, r, dH);
    else memset(dH, 0, sizeof(double) * 3 * (size_t)M);
    for (int p = 0; p < M; ++p) {
        const double Ry = R[M + p];
        for (int a = 0; a < 3; ++a) {
            const int i = a * M + p;
            R[i] = m->decay[p] * R[i] + m->h[p] * dH[i] + m->w[p] * Z[i];
        }
        R[p] += shear * m->g[p] * Ry;
    }
    free(r); free(dH);
}

/* One Euler step of the bead-position scheme (Eqs. b3-b5, btum) with the
 * bead noise z given: r_n += dtau (F_n + shear y_n x) + sqrt(2 T* dtau) z_n. */
void orc_euler_step_z(const orc_model *m, const double *z, double shear, double *r)
{
    const int M = m->M;
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    orc_full_force(m, r, F);
    const double amp = sqrt(2.0 * m->Tstar * m->dtau);
    for (int n = 0; n < M; ++n) F[n] += shear * r[M + n];
    for (int i = 0; i < 3 * M; ++i) r[i] += m->dtau * F[i] + amp * z[i];
    free(F);
}

/* ------------------------------------------------------------------------ */
/* Batched runners (OpenMP over chains)                                       */
/* ------------------------------------------------------------------------ */

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Advance C chains (R[c][3][M], p = 0 included) through nsteps mode-space
 * steps; chain c draws the noise of (seed, jobs[c], step0 + s, bead, tag 0). */
int orc_run_modes(const orc_model *m, int C, uint32_t seed, const uint32_t *jobs,
                  int64_t step0, int64_t nsteps, double shear, int coupling,
                  double *R, int nthreads)
{
    const int M = m->M;
    set_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < C; ++c) {
        double *z = (double *)malloc(sizeof(double) * 3 * (size_t)M);
        double *Rc = R + (size_t)c * 3 * M;
        for (int64_t s = 0; s < nsteps; ++s) {
            orc_bead_normals(seed, jobs[c], step0 + s, 0u, M, z);
            orc_mode_step_z(m, z, shear, coupling, Rc);
        }
        free(z);
    }
    return 0;
}

/* Same with mode-keyed noise: chain c draws Z of (seed, jobs[c], step0 + s,
 * mode, tag 2) by orc_mode_normals and takes it as the mode noise directly. */
int orc_run_modes_mk(const orc_model *m, int C, uint32_t seed, const uint32_t *jobs,
                     int64_t step0, int64_t nsteps, double shear, int coupling,
                     double *R, int nthreads)
{
    const int M = m->M;
    set_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < C; ++c) {
        double *Z = (double *)malloc(sizeof(double) * 3 * (size_t)M);
        double *Rc = R + (size_t)c * 3 * M;
        for (int64_t s = 0; s < nsteps; ++s) {
            orc_mode_normals(seed, jobs[c], step0 + s, M, Z);
            orc_mode_step_Zm(m, Z, shear, coupling, Rc);
        }
        free(Z);
    }
    return 0;
}

/* Same, for the bead-position Euler scheme on r[c][3][M]. */
int orc_run_euler(const orc_model *m, int C, uint32_t seed, const uint32_t *jobs,
                  int64_t step0, int64_t nsteps, double shear, double *r, int nthreads)
{
    const int M = m->M;
    set_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < C; ++c) {
        double *z = (double *)malloc(sizeof(double) * 3 * (size_t)M);
        double *rc = r + (size_t)c * 3 * M;
        for (int64_t s = 0; s < nsteps; ++s) {
            orc_bead_normals(seed, jobs[c], step0 + s, 0u, M, z);
            orc_euler_step_z(m, z, shear, rc);
        }
        free(z);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Starting conformations                                                     */
/* ------------------------------------------------------------------------ */

/* Straight-rod ground state of Eq. a2: the bond lengths l_n solve
 * dH'/dl_n = 0, i.e. l_n - nu (l_{n-1} + l_{n+1}) = 1, l_0 = l_{N+1} = 0. */
void orc_ground_bonds(const orc_model *m, double *l /* [N] */)
{
    const int N = m->M - 1;
    const double nu = m->nu;
    /* Thomas algorithm on the tridiagonal system (1 on the diagonal, -nu off it). */
    double *cp = (double *)malloc(sizeof(double) * N);
    double *dp = (double *)malloc(sizeof(double) * N);
    cp[0] = -nu; dp[0] = 1.0;
    for (int i = 1; i < N; ++i) {
        const double den = 1.0 + nu * cp[i - 1];
        cp[i] = -nu / den;
        dp[i] = (1.0 + nu * dp[i - 1]) / den;
    }
    l[N - 1] = dp[N - 1];
    for (int i = N - 2; i >= 0; --i) l[i] = dp[i] - cp[i] * l[i + 1];
    free(cp); free(dp);
}

/* Approximately equilibrated start of one chain (the paper leaves this open):
 *  1. bond lengths l ~ Normal(l0, T* (I - nu A)^-1): the straight-rod ground
 *     state plus the exact Gaussian of the quadratic stretching energy;
 *  2. tangents t_1 uniform on the sphere, t_n | t_{n-1} von Mises-Fisher with
 *     concentration nu l_{n-1} l_n / T* (the exact conditional of the bending
 *     term of Eq. a2 given the lengths);
 *  3. r_n = sum_{k<=n} l_k t_k, centre of mass moved to the origin, R = phi^T r.
 * Random numbers: counter (0, 0, k, 1); k = 0 draws t_1, k = n the bond n. */
void orc_equilibrium_start(const orc_model *m, uint32_t seed, uint32_t job, double *R)
{
    const int M = m->M, N = M - 1;
    const double nu = m->nu, T = m->Tstar;
    double *l0 = (double *)malloc(sizeof(double) * N);
    double *eps = (double *)malloc(sizeof(double) * N);
    double *x = (double *)malloc(sizeof(double) * N);
    double *Ld = (double *)malloc(sizeof(double) * N);   /* Cholesky diagonal */
    double *Lo = (double *)malloc(sizeof(double) * N);   /* Cholesky sub-diagonal */
    double *r = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    uint32_t (*bits)[4] = malloc(sizeof(uint32_t[4]) * (size_t)M);
    const uint32_t key[2] = {seed, job};
    for (int k = 0; k < M; ++k) {
        const uint32_t ctr[4] = {0u, 0u, (uint32_t)k, 1u};
        orc_philox4x32_10(ctr, key, bits[k]);
    }
    orc_ground_bonds(m, l0);
    for (int n = 1; n <= N; ++n)
        eps[n - 1] = sqrt(-2.0 * log(orc_u01(bits[n][0]))) * cos(2.0 * ORC_PI * orc_u01(bits[n][1]));
    /* (I - nu A) = L L^T, L lower bidiagonal; x = L^-T eps has covariance (I - nu A)^-1. */
    Ld[0] = 1.0; Lo[0] = 0.0;
    for (int i = 1; i < N; ++i) {
        Lo[i] = -nu / Ld[i - 1];
        Ld[i] = sqrt(1.0 - Lo[i] * Lo[i]);
    }
    x[N - 1] = eps[N - 1] / Ld[N - 1];
    for (int i = N - 2; i >= 0; --i) x[i] = (eps[i] - Lo[i + 1] * x[i + 1]) / Ld[i];
    const double sT = sqrt(T);
    /* first tangent: uniform on the sphere */
    double t[3];
    {
        const double cth = 2.0 * orc_u01(bits[0][0]) - 1.0;
        const double sth = sqrt((1.0 - cth) * (1.0 + cth));
        const double ph = 2.0 * ORC_PI * orc_u01(bits[0][1]);
        t[0] = sth * cos(ph); t[1] = sth * sin(ph); t[2] = cth;
    }
    r[0] = r[M] = r[2 * M] = 0.0;
    double lprev = 0.0;
    for (int n = 1; n <= N; ++n) {
        const double ln = l0[n - 1] + sT * x[n - 1];
        if (n >= 2 && T > 0.0) {
            const double kap = nu * lprev * ln / T;
            const double U = orc_u01(bits[n][2]);
            const double cth = 1.0 + log(U + (1.0 - U) * exp(-2.0 * kap)) / kap;
            const double sth = sqrt(fmax(0.0, (1.0 - cth) * (1.0 + cth)));
            const double ps = 2.0 * ORC_PI * orc_u01(bits[n][3]);
            /* orthonormal pair perpendicular to t (Duff et al., JCGT 2017) */
            const double sg = copysign(1.0, t[2]);
            const double a = -1.0 / (sg + t[2]);
            const double b = t[0] * t[1] * a;
            const double e1[3] = {1.0 + sg * t[0] * t[0] * a, sg * b, -sg * t[0]};
            const double e2[3] = {b, sg + t[1] * t[1] * a, -t[1]};
            double tn[3];
            for (int k = 0; k < 3; ++k)
                tn[k] = cth * t[k] + sth * (cos(ps) * e1[k] + sin(ps) * e2[k]);
            const double nn = sqrt(tn[0] * tn[0] + tn[1] * tn[1] + tn[2] * tn[2]);
            for (int k = 0; k < 3; ++k) t[k] = tn[k] / nn;
        }
        for (int k = 0; k < 3; ++k) r[k * M + n] = r[k * M + n - 1] + ln * t[k];
        lprev = ln;
    }
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int n = 0; n < M; ++n) s += r[k * M + n];
        s /= M;
        for (int n = 0; n < M; ++n) r[k * M + n] -= s;
    }
    orc_beads_to_modes(m, r, R);
    for (int k = 0; k < 3; ++k) R[k * M] = 0.0;   /* centre of mass exactly at the origin */
    free(l0); free(eps); free(x); free(Ld); free(Lo); free(r); free(bits);
}

/* ------------------------------------------------------------------------ */
/* Observables (Sec. 5B)                                                      */
/* ------------------------------------------------------------------------ */

/* From the mode state of one chain: out[0] = |L|^2 with L = r_N - r_0,
 * out[1] = |u_m|^2 of the middle bond m = ceil(N/2), out[2] = |r_m - r_cm|^2 of
 * the middle bead m = floor(N/2), out[3..5] = r_cm. */
void orc_observables(const orc_model *m, const double *R, double *out)
{
    const int M = m->M, N = M - 1;
    double *r = (double *)malloc(sizeof(double) * 3 * (size_t)M);
    orc_modes_to_beads(m, R, r);
    double cm[3];
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int n = 0; n < M; ++n) s += r[a * M + n];
        cm[a] = s / M;
    }
    const int mb = (N + 1) / 2, mm = N / 2;
    double L2 = 0, u2 = 0, d2 = 0;
    for (int a = 0; a < 3; ++a) {
        const double L = r[a * M + N] - r[a * M];
        const double u = r[a * M + mb] - r[a * M + mb - 1];
        const double d = r[a * M + mm] - cm[a];
        L2 += L * L; u2 += u * u; d2 += d * d;
    }
    out[0] = L2; out[1] = u2; out[2] = d2;
    out[3] = cm[0]; out[4] = cm[1]; out[5] = cm[2];
    free(r);
}

/* ------------------------------------------------------------------------ */
/* Metropolis Monte Carlo in the mode representation (Sec. 5A)               */
/* ------------------------------------------------------------------------ */

/* Scaled energy H' of Eq. a2 from the bond vectors u[a*N + (n-1)], n = 1..N. */
static double energy_of_bonds(int N, double nu, const double *u)
{
    double e = 0.0;
    for (int n = 0; n < N; ++n) {
        const double ux = u[n], uy = u[N + n], uz = u[2 * N + n];
        const double len = sqrt(ux * ux + uy * uy + uz * uz);
        e += 0.5 * (len - 1.0) * (len - 1.0);
        if (n >= 1) e -= nu * (ux * u[n - 1] + uy * u[N + n - 1] + uz * u[2 * N + n - 1]);
    }
    return e;
}

/* Bonds of a mode state, u_n = sum_p chi_{n,p} R_p (Eq. e5). */
static void bonds_of_modes(const orc_model *m, const double *R, double *u)
{
    const int M = m->M, N = M - 1;
    for (int a = 0; a < 3; ++a)
        for (int n = 1; n <= N; ++n) {
            double s = 0.0;
            for (int p = 0; p < M; ++p) s += m->chi[(size_t)(n - 1) * M + p] * R[a * M + p];
            u[a * N + n - 1] = s;
        }
}

/* The equilibrium benchmark of Sec. 5A: Monte Carlo in the mode amplitudes
 * with large moves for the slow modes and small moves for the fast ones.
 * One sweep visits every internal mode p = 1..N and axis alpha in order and
 * proposes R_p^alpha += delta, delta uniform on (-s_p, s_p); the bonds then
 * change by chi_{n,p} delta along alpha (Eq. e5), the energy H' is
 * recomputed from them (Eq. a2) and the move is accepted with probability
 * min(1, exp(-(H'_new - H'_old)/T*)).  The map R -> u is linear with a
 * constant Jacobian, so the chain samples exp(-H'/T*) over bond space.
 * The centre-of-mass mode p = 0 does not enter H' and is left unchanged.
 * Random numbers: Philox counter (sweep_lo, sweep_hi, 3(p-1)+alpha, 3); word 0
 * draws delta, word 1 the acceptance uniform.
 *   acc[p]   incremented once per accepted move of mode p (any axis);
 *   obs[k]   if non-NULL, after every sweep adds observables (orc_observables)
 *            0..2, i.e. |L|^2, |u_m|^2 and |r_m - r_cm|^2, and obs[3] += 1. */
void orc_mc_sweeps(const orc_model *m, uint32_t seed, uint32_t job, int64_t sweep0,
                   int64_t n_sweeps, const double *step, double *R, int64_t *acc, double *obs)
{
    const int M = m->M, N = M - 1;
    const double T = m->Tstar;
    double *u = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *un = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    const uint32_t key[2] = {seed, job};
    for (int64_t s = 0; s < n_sweeps; ++s) {
        const int64_t sw = sweep0 + s;
        bonds_of_modes(m, R, u);            /* fresh every sweep: no drift from updates */
        double e = energy_of_bonds(N, m->nu, u);
        for (int p = 1; p <= N; ++p)
            for (int a = 0; a < 3; ++a) {
                const uint32_t ctr[4] = {(uint32_t)((uint64_t)sw & 0xffffffffu),
                                         (uint32_t)((uint64_t)sw >> 32),
                                         (uint32_t)(3 * (p - 1) + a), 3u};
                uint32_t x[4];
                orc_philox4x32_10(ctr, key, x);
                const double delta = step[p] * (2.0 * orc_u01(x[0]) - 1.0);
                memcpy(un, u, sizeof(double) * 3 * (size_t)N);
                for (int n = 1; n <= N; ++n) un[a * N + n - 1] += m->chi[(size_t)(n - 1) * M + p] * delta;
                const double en = energy_of_bonds(N, m->nu, un);
                const double de = en - e;
                if (de <= 0.0 || orc_u01(x[1]) < exp(-de / T)) {
                    R[a * M + p] += delta;
                    memcpy(u, un, sizeof(double) * 3 * (size_t)N);
                    e = en;
                    if (acc) acc[p] += 1;
                }
            }
        if (obs) {
            double o[6];
            orc_observables(m, R, o);
            obs[0] += o[0]; obs[1] += o[1]; obs[2] += o[2]; obs[3] += 1.0;
        }
    }
    free(u); free(un);
}

/* orc_mc_sweeps for C independent chains (OpenMP over chains): chain c uses
 * job jobs[c], its state R[c][3][M], acceptance counts acc[c][M] and
 * observable sums obs[c][4] (either may be NULL). */
int orc_run_mc(const orc_model *m, int C, uint32_t seed, const uint32_t *jobs, int64_t sweep0,
               int64_t n_sweeps, const double *step, double *R, int64_t *acc, double *obs,
               int nthreads)
{
    const int M = m->M;
    set_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < C; ++c)
        orc_mc_sweeps(m, seed, jobs[c], sweep0, n_sweeps, step, R + (size_t)c * 3 * M,
                      acc ? acc + (size_t)c * M : NULL, obs ? obs + (size_t)c * 4 : NULL);
    return 0;
}
