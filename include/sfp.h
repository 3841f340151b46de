/*
 * sfp.h -- C ABI of the GB300 mode-space Langevin integrator for the
 * extensible bead-spring model of semiflexible polymers (Panja, Barkema,
 * van Leeuwen, "Efficient simulation of semiflexible polymers",
 * arXiv:1411.3487).
 *
 * One batch = many independent chains (no hydrodynamics, Sec. 1), each with
 * its own length, step size, shear rate and noise key.  Every call returns
 * SFP_OK (0) or a negative SFP_E* code; sfp_last_error() then holds a
 * one-line message for the calling thread.
 *
 * Units at this boundary: nm, ps, 1/s.  Inside, the paper's scaled units
 * (Sec. 3, Eqs. b3-b5): lengths in d = a(1-2 nu), time in xi/lambda, so that
 * t = c tau with c = T* (1-2nu)^2 a^2 xi / kT (Eq. g2).
 *
 * Ownership: the caller owns every host buffer it passes and may reuse it as
 * soon as the call returns.  A batch owns all device memory it allocates and
 * frees it in sfp_destroy().  Device work is queued on the batch's stream;
 * only sfp_observe, sfp_probe, sfp_save and the sfp_set_* calls synchronise it.
 *
 * Packed per-chain arrays: for chains c = 0..C-1 (in the order given to
 * sfp_create) with M_c beads, chain c's block is [3][M_c] (axis-major, index
 * contiguous) and starts at offset 3 * sum_{c' < c} M_{c'} elements.
 */
#ifndef SFP_H
#define SFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SFP_OK          0
#define SFP_EINVAL     -1   /* bad argument (see sfp_last_error) */
#define SFP_ENOMEM     -2   /* device allocation failed or exceeds the HBM budget */
#define SFP_ECUDA      -3   /* a CUDA runtime call failed */
#define SFP_ETIMEDOUT  -4   /* a bounded device wait gave up (every wait of the
                               tensor-core kernels is limited to 1 s; the kernel
                               then returns and the context stays usable; with
                               SFP_TEST_STALL=1 in the environment the fused
                               step stalls on purpose, to test this) */
#define SFP_ENONFINITE -5   /* a chain's state became non-finite */
#define SFP_ENOTSUP    -6   /* valid request that the library does not support */

/* ---- model parameters (Eqs. a1-a3, Sec. 2A, Sec. 7B) --------------------- */
typedef struct sfp_params {
    /* Stretching and bending stiffness lambda, kappa of Eq. a1 (pN/nm).
     * If lambda <= 0 the dimensionless pair (T_star, nu) below is used. */
    double lambda_pN_per_nm;
    double kappa_pN_per_nm;
    double a_nm;             /* mean bead spacing a = b d (Sec. 2; 0.33 nm for dsDNA) */
    double xi_kg_per_s;      /* bead friction xi (Eq. g1: 1.91e-12 kg/s) */
    double kT_pN_nm;         /* thermal energy (4.089 pN nm at 23 C, Sec. 7B) */
    double T_star;           /* T* = kT / (lambda d^2), used when lambda <= 0 */
    double nu;               /* nu = kappa / lambda, 0 < nu < 1/2 (Sec. 2) */
    /* a^2 xi / kT in ps (Eq. factor).  > 0: used as given (52.0 is the
     * printed value, which reproduces Table 2); 0: computed from a, xi, kT. */
    double a2xi_over_kT_ps;
} sfp_params;

/* Fill the paper's dsDNA parameter set (Sec. 2A, Sec. 7B): T* = 0.034,
 * nu = 0.35, a = 0.33 nm, xi = 1.91e-12 kg/s, kT = 4.089 pN nm, and the
 * printed a^2 xi / kT = 52.0 ps.  Host only; never fails for p != NULL. */
int sfp_params_dsdna(sfp_params *p);

/* Derived constants (host only, no GPU needed):
 * out[0] = T*, out[1] = nu, out[2] = c (ps per unit of scaled time, Eq. g2),
 * out[3] = d (nm), out[4] = b = 1/(1-2nu) (Eq. a3), out[5] = l_p/a = b^2 nu/T*
 * (Eq. a3), out[6] = lambda (pN/nm), out[7] = kappa (pN/nm).
 * SFP_EINVAL if nu is outside (0, 1/2) (Sec. 2) or a value is non-positive. */
int sfp_derive(const sfp_params *p, double out[8]);

/* ---- chains --------------------------------------------------------------- */
typedef struct sfp_chain_desc {
    int32_t  n_beads;          /* N+1 beads = basepairs (Sec. 2A); 3..4096 */
    int32_t  reserved;         /* must be 0 */
    double   dt_ps;            /* step in ps; used when dtau <= 0 (Table 2) */
    double   dtau;             /* step in scaled time; > 0 takes precedence */
    double   shear_rate_per_s; /* gamma-dot of Eq. btum (flow v = gamma y x); 0 = none */
    uint64_t job_id;           /* Philox key word of this chain's noise; < 2^32 */
} sfp_chain_desc;

/* Arithmetic of the step.  In every mode the centre of mass, its MSD windows
 * and the sampled sums are FP64 on the GPU.
 * SFP_FP32 (= SFP_MIXED_TF32)
 *                 FP32 state, forces and update; the two transforms run on the
 *                 tensor cores (tcgen05, kind::tf32) as a three-pass TF32
 *                 hi/lo split (A_hi B_lo + A_lo B_hi + A_hi B_hi) with FP32
 *                 accumulation, which keeps FP32 trajectory accuracy (fused
 *                 step for 64/128/256/512 beads, staged otherwise).  The name
 *                 says what the state is; the transforms are TF32x3.
 * SFP_FP64        FP64 throughout (CUDA cores).
 * SFP_MIXED_BF16  as SFP_FP32, but the transforms as a three-pass BF16 hi/lo
 *                 split (kind::f16, BF16 A and B), FP32 accumulate: hi and lo
 *                 carry about 16 bits of each operand.  Both the fused step
 *                 and the staged kernels form DeltaH = chi^T v in bond form
 *                 (Eq. e11); trajectories stay within 1e-5 of the FP64 oracle
 *                 after 1000 steps.
 * SFP_MIXED_BF16_2  as SFP_MIXED_BF16 with two passes, A_lo B_hi + A_hi B_hi:
 *                 the state operand (R, v, z) keeps its hi/lo split, the
 *                 tables (chi, h chi, w phi) are rounded to BF16 (about 8
 *                 bits), so a third fewer MMAs; the error against the FP64
 *                 oracle is about 1e-3 per step's transform, well above the
 *                 FP32 tolerance (stated per observable by the precision test).
 * SFP_FP32_SIMT   FP32 throughout on the CUDA cores: the plain path. */
enum { SFP_FP32 = 0, SFP_MIXED_TF32 = 0, SFP_FP64 = 1, SFP_MIXED_BF16 = 2, SFP_MIXED_BF16_2 = 3,
       SFP_FP32_SIMT = 4 };

typedef struct sfp_batch sfp_batch;   /* opaque */

/* Create a batch of n_chains chains.  Chains are grouped internally by
 * (n_beads, dtau); each group gets its own tables (Eqs. c8, c9, e9, d3, d6,
 * f2).  The initial state is the straight ground-state rod along x with its
 * centre of mass at the origin; call sfp_init_equilibrium or sfp_set_* next.
 *   seed        Philox key word 0 (< 2^32); job_id is key word 1.
 *   cuda_stream cudaStream_t to queue work on (NULL = legacy default stream).
 *   hbm_budget_bytes  upper bound on device memory this batch may hold
 *               (0 = no bound); exceeding it returns SFP_ENOMEM.
 * On failure *out is set to NULL and nothing is leaked. */
int sfp_create(const sfp_params *params, const sfp_chain_desc *chains, int32_t n_chains,
               uint64_t seed, int32_t precision, void *cuda_stream,
               size_t hbm_budget_bytes, sfp_batch **out);

/* Replace every chain's conformation by an approximately equilibrated one
 * (the paper leaves the start open): bond lengths from the Gaussian of the
 * stretching energy about the straight-rod ground state of Eq. a2, tangents
 * as a von Mises-Fisher chain with concentration nu l_{n-1} l_n / T*, centre
 * of mass at the origin.  Philox counter (0, 0, k, 1).  Then runs
 * burn_in_steps ordinary steps.  Resets step counters to 0 first. */
int sfp_init_equilibrium(sfp_batch *b, int64_t burn_in_steps);

/* Set the state from host FP64 arrays, packed per chain as [3][M_c].
 * sfp_set_modes takes mode amplitudes R_p (p = 0..N, Eq. c1) in scaled
 * units, with R_0 = sqrt(N+1) r_cm; sfp_set_positions takes absolute bead
 * positions in nm.  Step counters are left unchanged.  Synchronous.  With one
 * length group and a page-locked buffer (e.g. cudaHostAlloc), sfp_set_modes
 * reads the caller's buffer from the GPU directly (no staging copy); the
 * same holds for SFP_OBS_MODES of sfp_observe. */
int sfp_set_modes(sfp_batch *b, const double *host_modes, size_t n_doubles);
/* sfp_set_modes from FP32 amplitudes (same layout and units, n_floats values):
 * half the host traffic; the SFP_FP32 / mixed state is FP32 already, so only
 * R_0 (the centre of mass, carried in FP64) is rounded.  SFP_EINVAL for a NULL
 * argument or too few values. */
int sfp_set_modes_f32(sfp_batch *b, const float *host_modes, size_t n_floats);
int sfp_set_positions(sfp_batch *b, const double *host_pos_nm, size_t n_doubles);

/* Set every chain's step counter (the Philox counter of its next step). */
int sfp_set_step(sfp_batch *b, int64_t step);

/* Advance every chain by n_steps mode-space steps (Sec. 4):
 *   bond vectors u = chi R (Eq. e5); DeltaH = chi^T v from the bond forces
 *   (Eq. e11); bead noise z ~ N(0,1) keyed by (seed, job_id, step, bead, axis)
 *   (see SFP_PROBE_NOISE) and projected (Eq. c4);
 *   R_p <- e^{-zeta_p dtau} R_p + h_p DeltaH_p + w_p Z_p (Eqs. d3, d6, f2);
 *   shear adds gamma g_p R^y_p to R^x_p (Eq. btum); the centre of mass
 *   (p = 0) is carried in FP64.
 * Asynchronous on the batch's stream.  SFP_EINVAL for n_steps < 0. */
int sfp_step(sfp_batch *b, int64_t n_steps);

/* Observables, copied to host_out (synchronises the stream).
 *   SFP_OBS_MODES      FP64 packed [3][M_c], scaled units, R_0 = sqrt(M) r_cm
 *   SFP_OBS_MODES_F32  the same rounded to FP32 (half the bytes; written
 *                      directly like SFP_OBS_MODES into a page-locked buffer)
 *   SFP_OBS_POSITIONS  FP64 packed [3][M_c], absolute bead positions in nm
 *   SFP_OBS_COM        FP64 [C][3] centre of mass in nm
 *   SFP_OBS_STEP       int64 [C] step counters
 *   SFP_OBS_SHAPE      FP64 [C][4] per chain: |L|^2 (L = r_N - r_0), |u_m|^2 of
 *                      the middle bond m = ceil(N/2), |r_m - r_cm|^2 of the
 *                      middle bead m = floor(N/2) (Sec. 5B, observables
 *                      i-iii at this instant), all in nm^2, and the
 *                      simulated time t = c tau in ps
 * Accumulators of sfp_set_sampling (SFP_EINVAL before its first call):
 *   SFP_OBS_ACCUM      FP64 [C][4] per chain: sums over samples of the three
 *                      SFP_OBS_SHAPE quantities (nm^2) and the sample count;
 *                      their ratio is the equilibrium value Q(0) of the
 *                      paper's observables i-iii (Sec. 5B)
 *   SFP_OBS_MODE_POWER FP64 packed [3][M_c]: sums over samples of (R_p^alpha)^2
 *                      in scaled units (R_0 = sqrt(M) r_cm)
 *   SFP_OBS_COM_MSD    FP64 [C][L][2] per chain and lag (L lags of sfp_set_msd_lags,
 *                      by default 4: 1, 10, 100, 1000 sampling intervals): sum
 *                      of |r_cm(t) - r_cm(t - lag)|^2 (nm^2, FP64 centre of
 *                      mass, non-overlapping windows) and the number of
 *                      windows; ratio / (6 t_lag) estimates the diffusion
 *                      coefficient kT/((N+1) xi) of Sec. 7B
 *   SFP_OBS_MID_MSD    FP64 [C][L][2]: the same windows for the middle bead
 *                      m = floor(N/2) relative to the centre of mass: sum of
 *                      |(r_m - r_cm)(t) - (r_m - r_cm)(t - lag)|^2 (nm^2) and the
 *                      number of windows; their ratio is the mean-square
 *                      displacement Q(t_lag) of observable iii of Sec. 5B
 *   SFP_OBS_E2E_MSD    FP64 [C][L][2]: the same windows for the end-to-end vector
 *                      L: sum of |L(t) - L(t - lag)|^2 (nm^2) and the windows;
 *                      for a stationary chain <L(t).L(0)> = <|L|^2> - ratio / 2,
 *                      the time autocorrelation of observable i (Sec. 5B)
 *   SFP_OBS_BOND_MSD   FP64 [C][L][2]: the same for the middle bond u_m
 *                      (observable ii)
 *   SFP_OBS_E2E2_MEAN  FP64 [C]: mean |L|^2 over the samples (nm^2), the
 *                      equilibrium <|L|^2> of observable i (Sec. 5B)
 *   SFP_OBS_MODE_VAR   FP64 packed [3][M_c]: mean of (R_p^alpha)^2 over the
 *                      samples (scaled units; equipartition gives about
 *                      T* / zeta_p for the transverse part, Sec. 4)
 * bytes must be at least the size of the requested array. */
enum { SFP_OBS_MODES = 0, SFP_OBS_POSITIONS = 1, SFP_OBS_COM = 2, SFP_OBS_STEP = 3,
       SFP_OBS_SHAPE = 4, SFP_OBS_ACCUM = 5, SFP_OBS_MODE_POWER = 6, SFP_OBS_COM_MSD = 7,
       SFP_OBS_MID_MSD = 8, SFP_OBS_E2E2_MEAN = 9, SFP_OBS_MODE_VAR = 10, SFP_OBS_E2E_MSD = 11,
       SFP_OBS_BOND_MSD = 12, SFP_OBS_MODES_F32 = 13 };
int sfp_observe(sfp_batch *b, int32_t what, void *host_out, size_t bytes);

/* Kernel path of the step (SFP_FP32_SIMT ignores it).
 *   SFP_PATH_FUSED   (default) chains of 64, 128, 256 or 512 beads take one
 *                    kernel per step and group: inverse transform, bond force,
 *                    noise, forward transform and mode update in one launch
 *                    with the intermediates kept on chip (TMEM and shared
 *                    memory; at 512 beads a tile runs on a cluster of two
 *                    CTAs, one per half of the bonds and modes); other lengths
 *                    take the staged path.  SFP_FP64 chains of up to 2048 beads
 *                    take one CUDA-core kernel per chunk of steps, a CTA per
 *                    chain with its state in shared memory between steps.
 *   SFP_PATH_STAGED  one kernel per stage; keeps the intermediate arrays, so
 *                    sfp_probe works after the step.
 * Both give the same trajectory within FP32 rounding.  SFP_EINVAL otherwise. */
enum { SFP_PATH_FUSED = 0, SFP_PATH_STAGED = 1 };
int sfp_set_path(sfp_batch *b, int32_t path);

/* Launch plan of sfp_step.
 * sfp_set_graph(b, 1): each chunk of steps (up to 1024, or 64 when a group
 * takes the staged kernels; chunks end at observable samples) is captured
 * once into a CUDA graph on an internal stream and replayed on the batch's
 * stream; off with stage timing and for the Euler integrator.  A batch of
 * several length groups runs each group on its own stream, forked from and
 * joined back into the batch's stream, so the groups share the GPU.
 * sfp_autotune(b, trial_steps, out): chooses the chains per tile of every
 * fused group (4..40, a multiple of 4) by timing candidates for trial_steps
 * steps, alone and together; the state, noise counters and trajectory are
 * restored after every trial (it allocates a temporary copy of the state
 * outside the HBM budget).
 * out, if not NULL, receives each group's choice (0 for staged groups), in
 * order of first appearance of each (n_beads, dtau) in the chain list. */
int sfp_set_graph(sfp_batch *b, int32_t enable);
/* Grouped launch (default on): the length groups on the fused step (at most
 * one group each of 64, 128, 256 and 512 beads; any others keep launches of
 * their own) advance together in one launch of clusters of two CTAs: a
 * cluster runs either one 512-bead tile on both CTAs or two tiles of the other
 * lengths, one per CTA, and clusters start in order of tile length (longest
 * first) as SMs free up.  The trajectories are those of one launch per group.
 * Off: one launch per group, each on its own stream.  Host only. */
int sfp_set_grouped(sfp_batch *b, int32_t enable);
int sfp_autotune(sfp_batch *b, int32_t trial_steps, int32_t *chains_per_tile);

/* Integrator of sfp_step.
 *   SFP_INTEGRATOR_MODES  the mode-space step of Sec. 4 (default).
 *   SFP_INTEGRATOR_EULER  the default bead-position Euler scheme of Sec. 3A
 *                         (Eqs. b3-b5): r_n += dtau (F_n + gamma y_n x)
 *                         + sqrt(2 T* dtau) z_n with the full force of Eq. a2,
 *                         stable only for small dtau (about 0.1, Sec. 3A), with
 *                         the same bead noise z_n as the mode-space step.  It
 *                         runs on the bond vectors (FP32 keeps the small
 *                         increments) and the FP64 centre of mass; each
 *                         sfp_step call converts modes -> bonds -> modes once.
 *                         Up to 4096 beads; probes are not kept.
 * SFP_EINVAL for an unknown value. */
enum { SFP_INTEGRATOR_MODES = 0, SFP_INTEGRATOR_EULER = 1 };
int sfp_set_integrator(sfp_batch *b, int32_t integrator);

/* Noise keying of the mode-space step (Eq. c4: the bead noise enters the mode
 * equations only through Z = phi^T z; phi is orthonormal, so the projection of
 * iid normals is iid normal again).
 *   SFP_NOISE_BEADS  (default) the bead normals z of (seed, job, step, tag 0)
 *                    are drawn and projected, Z = phi^T z: the same noise as
 *                    the bead-position Euler scheme, so the two integrators can
 *                    be compared path by path.
 *   SFP_NOISE_MODES  Z itself is drawn per mode, normal 3 p + alpha of Philox
 *                    call (3 p + alpha) / 4 under tag 2: the same distribution,
 *                    a different stream; the projection's contraction (a third
 *                    of the forward transform) is skipped.  The fused step takes
 *                    it at 64, 128 and 256 beads with three passes (the noise
 *                    warps draw Z one step ahead into a buffer of two steps,
 *                    8 C M bytes, allocated here and counted against the
 *                    budget); 512-bead and SFP_MIXED_BF16_2 groups then run on
 *                    the staged kernels, and the grouped launch is off.  The
 *                    Euler integrator and sfp_step_noalloc always draw bead
 *                    noise.  Host only; SFP_EINVAL for an unknown value. */
enum { SFP_NOISE_BEADS = 0, SFP_NOISE_MODES = 1 };
int sfp_set_noise(sfp_batch *b, int32_t keying);

/* Observable sampling (Sec. 5B).  every_steps > 0 clears the accumulators of
 * SFP_OBS_ACCUM, SFP_OBS_MODE_POWER and SFP_OBS_COM_MSD, takes sample 0 of the
 * current state at once, and from then on one sample after every every_steps
 * steps of sfp_step (a small kernel on the batch's stream; the first call
 * allocates about 8 (3 M + 16) bytes per chain).  every_steps = 0 stops
 * sampling and keeps the sums readable.  Accumulators are not part of a
 * checkpoint (sfp_save).  SFP_EINVAL for every_steps < 0. */
int sfp_set_sampling(sfp_batch *b, int32_t every_steps);

/* Lags of the SFP_OBS_COM_MSD, _MID_MSD, _E2E_MSD and _BOND_MSD windows, in sampling
 * intervals: n_lags = 1..8 values, each >= 1 (default 1, 10, 100, 1000).  The
 * list takes effect at the next sfp_set_sampling(b, every_steps > 0), which
 * clears the windows; from then on those observables have n_lags rows per
 * chain.  Host only.  SFP_EINVAL otherwise. */
int sfp_set_msd_lags(sfp_batch *b, int32_t n_lags, const int32_t *lags);

/* Intermediate arrays of the most recent step, FP64 packed [3][M_c] in scaled
 * units, for checking each stage on its own:
 *   SFP_PROBE_BONDS  bond vectors u_n = r_n - r_{n-1} = sum_p chi_{n,p} R_p
 *                    (Eq. e5) at index n = 1..N; index 0 holds 0
 *   SFP_PROBE_FORCE  bond forces v_n = u_n (1/|u_n| - (1-2nu)) at n = 1..N,
 *                    index 0 holds 0, so that chi^T v = DeltaH (Eq. e11)
 *   SFP_PROBE_NOISE  bead normals z of that step (Eq. b5, unit variance):
 *                    the normal of bead n, axis alpha is number k = 3n + alpha
 *                    of the step, value k mod 4 of Philox call k / 4 (counter
 *                    (step_lo, step_hi, k / 4, 0), key (seed, job_id);
 *                    Box-Muller on the word pairs (0,1) and (2,3))
 *   SFP_PROBE_DH     chi^T v = DeltaH_p (Eq. e11)
 *   SFP_PROBE_ZMODE  phi^T z = Z_p (Eq. c4)
 * SFP_EINVAL if no step has run since the batch was created or its state set,
 * or if the last step ran on SFP_PATH_FUSED (set SFP_PATH_STAGED first). */
enum { SFP_PROBE_BONDS = 0, SFP_PROBE_FORCE = 1, SFP_PROBE_NOISE = 2, SFP_PROBE_DH = 3,
       SFP_PROBE_ZMODE = 4 };
int sfp_probe(sfp_batch *b, int32_t what, void *host_out, size_t bytes);

/* Checkpoint / resume.  sfp_save writes the whole dynamic state (modes,
 * centre of mass, step counters) into host_buf; *needed receives the size
 * (host_buf may be NULL to query it).  sfp_load restores it into a batch
 * created with the same chains and precision.  Because the noise is
 * counter-based, a resumed run continues the same trajectory bit for bit. */
int sfp_save(sfp_batch *b, void *host_buf, size_t bytes, size_t *needed);
int sfp_load(sfp_batch *b, const void *host_buf, size_t bytes);

/* Number of chains, total beads, device bytes held, and kernel launches
 * issued by sfp_step so far (out[0..3]). */
int sfp_info(const sfp_batch *b, int64_t out[4]);

/* Stage timing.  While enabled, every sfp_step records CUDA events on the
 * batch's stream between its stage launches (inverse transform, bond force,
 * bead noise, forward transform, mode update); the noise kernel then runs in
 * line on the batch's stream instead of beside the inverse transform on a
 * stream of its own, and the length groups one after another.  Enabling clears
 * the totals.  sfp_stage_times synchronises the stream and writes the summed
 * device time in microseconds of [inverse, force, noise, forward, update,
 * whole step] over *n_group_steps recorded group-steps (one per length group
 * per step).  A fused step (SFP_PATH_FUSED) is one kernel: its whole time is
 * counted in the first entry and in the whole-step entry. */
int sfp_stage_timing(sfp_batch *b, int32_t enable);
int sfp_stage_times(sfp_batch *b, double out_us[6], int64_t *n_group_steps);

/* Free every device buffer of the batch (synchronises its stream). NULL is a no-op. */
int sfp_destroy(sfp_batch *b);

/* Last error message of the calling thread ("" if none). */
const char *sfp_last_error(void);

/* Raw Philox4x32-10 words computed on the GPU for counter (step_lo, step_hi,
 * i, tag) and key (seed, job), i = 0..count-1, into host_out[4*count].
 * For checking the device generator bit for bit; synchronous. */
int sfp_philox_words(uint32_t seed, uint32_t job, int64_t step, uint32_t tag,
                     int32_t count, uint32_t *host_out);

/* ---- serving: continuous batching of simulation jobs -----------------------
 * A server accepts jobs at any time (from any thread), keeps every running
 * chain's mode state on the GPU, and advances all running jobs together:
 * jobs of one (length, step size) share a pool of slots that one sfp_step call
 * per quantum advances, so a job that arrives while others run joins their
 * next launch.  Pools are created as jobs need them while the HBM budget
 * allows (a pool that does not fit is retried with half as many slots), and
 * idle pools of other shapes are released to make room; a job that does not
 * fit waits for running jobs to finish, and finishes with status SFP_ENOMEM
 * if even a one-slot pool cannot fit while nothing runs.  Each job starts from the equilibrium sampler of
 * sfp_init_equilibrium keyed by (seed, job_id), with its own step counter
 * from 0, so its result does not depend on the slot it ran in or on the other
 * jobs (noise keyed by (seed, job_id, step, bead)).  A job stops exactly
 * after its n_steps steps even inside a quantum.  One worker thread per
 * server issues all GPU work on the server's own stream. */
typedef struct sfp_server sfp_server;   /* opaque */

typedef struct sfp_server_config {
    uint64_t seed;               /* Philox key word 0 (< 2^32) */
    int32_t  precision;          /* any precision of sfp_create (SFP_MIXED_BF16 is fastest) */
    int32_t  slots_per_pool;     /* chains per pool (one pool per allocation) */
    int32_t  quantum_steps;      /* steps per round of the request loop */
    int32_t  keep_results;       /* 1: keep each job's final modes for sfp_server_result_modes */
    size_t   hbm_budget_bytes;   /* device memory all pools together may hold (0 = no bound) */
} sfp_server_config;

typedef struct sfp_job {
    int32_t  n_beads;            /* N+1 beads (Sec. 2A); 3..4096 */
    int32_t  reserved;           /* must be 0 */
    double   dt_ps;              /* step in ps; used when dtau <= 0 */
    double   dtau;               /* step in scaled time; > 0 takes precedence */
    double   shear_rate_per_s;   /* gamma-dot of Eq. btum; 0 = none */
    int64_t  n_steps;            /* steps to run (>= 0) */
    uint64_t job_id;             /* Philox key word 1 of this job; < 2^32 */
} sfp_job;

typedef struct sfp_job_result {
    uint64_t ticket;             /* as returned by sfp_server_submit */
    uint64_t job_id;
    int32_t  n_beads;
    int32_t  status;             /* SFP_OK or a negative SFP_E* code */
    int64_t  n_steps;
    double   submit_s, admit_s, finish_s;   /* server clock (s since sfp_server_create) */
    double   com_nm[3];          /* final centre of mass (nm) */
} sfp_job_result;

/* Defaults: seed 1, SFP_FP32, 512 slots per pool, quantum 64 steps, results
 * kept, no budget bound.  Host only. */
int sfp_server_config_default(sfp_server_config *cfg);
/* Start a server (and its worker thread) on the current CUDA device. */
int sfp_server_create(const sfp_params *params, const sfp_server_config *cfg, sfp_server **out);
/* Queue a job; thread-safe; never blocks on the GPU.  *ticket numbers jobs
 * from 0 in submission order.  SFP_EINVAL for a malformed job. */
int sfp_server_submit(sfp_server *s, const sfp_job *job, uint64_t *ticket);
/* Move up to max_results finished jobs into out (oldest first); *n_out gets
 * the count.  Non-blocking.  Returns the worker's error code if it stopped. */
int sfp_server_poll(sfp_server *s, sfp_job_result *out, int32_t max_results, int32_t *n_out);
/* Final mode amplitudes of a finished job, FP64 [3][n_beads] in scaled units
 * (R_0 = sqrt(n_beads) r_cm), when keep_results = 1. */
int sfp_server_result_modes(sfp_server *s, uint64_t ticket, double *host_modes, size_t n_doubles);
/* Block until no job is waiting or running, or timeout_s passes (SFP_ETIMEDOUT). */
int sfp_server_wait_idle(sfp_server *s, double timeout_s);
/* out[0..9]: jobs submitted, finished, waiting, running; device bytes held
 * by the server's pools (the library's fixed SFP_NOALLOC_SCRATCH_BYTES array,
 * resident on every device that loads the library, is outside both this count
 * and the HBM budget);
 * p50, p99 and max latency (finish - submit, s); server clock (s); bead-steps
 * of the finished jobs. */
int sfp_server_stats(sfp_server *s, double out[10]);
/* Stop the worker (running jobs are abandoned), free every pool. NULL is a no-op. */
int sfp_server_destroy(sfp_server *s);
/* Last error message of the calling thread for sfp_server_* calls. */
const char *sfp_server_last_error(void);

/* ---- allocation-free step -------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory: code running inside a host framework that
 * owns every device buffer (its own pool, or a fixed budget enforced by an
 * outside memory manager), and latency-critical loops where a cudaMalloc,
 * which may synchronise the whole device, would stall other streams.
 *
 * sfp_step_noalloc advances n_chains chains that live in caller-owned device
 * memory by n_steps steps of the plain FP32 CUDA-core path (the same kernels
 * and the same arithmetic as sfp_step on an SFP_FP32_SIMT batch).  It calls
 * no cudaMalloc, cudaFree or other allocating routine: its tables (phi,
 * phi^T and the per-mode coefficients, rebuilt on the device on every call)
 * and its scratch (bead positions, force and noise, mode-space force and
 * noise, step counters) live in one file-scope device array of
 * SFP_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU which loads the library
 * holds until the process exits.
 *   chain      n_beads, step (dtau, or dt_ps when dtau <= 0) and shear rate
 *              shared by all chains; chain c uses Philox key
 *              (seed, chain->job_id + c) and must keep job_id + c < 2^32.
 *   step0      step counter of the first step (the Philox counter), the
 *              same for every chain.
 *   modes_dev  FP32 device array [n_chains][3][n_beads] of mode amplitudes
 *              R_p in scaled units (in/out).  Entries p = 0 are ignored on
 *              input and set to 0: the centre of mass is com_dev.
 *   com_dev    FP64 device array [n_chains][3], centre of mass in scaled
 *              units (in/out).
 *   cuda_stream  the stream to queue the work on (NULL = legacy default).
 * Scratch needed: 4 * (3 M^2 + 4 M + 15 n_chains M) bytes plus
 * 24 * n_chains bytes (each piece rounded up to 256 bytes); a request that does
 * not fit returns SFP_EINVAL with the limit in sfp_last_error().
 * Every call looks up the array's device address on the current device with
 * cudaGetSymbolAddress (a host-side query, so a device reset does not leave a
 * stale address behind); make the first call on a device before any stream
 * capture, since it loads the library's device code there.  The array is not
 * part of any batch's or server's HBM budget or held-bytes count.  Every call
 * shares the one array, which keeps
 * the previous call's contents; calls whose work overlaps on the GPU (two
 * streams, or two host threads) race on it and must be serialised by the
 * caller.  Asynchronous on cuda_stream; non-finite states are not reported. */
#define SFP_NOALLOC_SCRATCH_BYTES (32u << 20)
int sfp_step_noalloc(const sfp_params *params, const sfp_chain_desc *chain, int32_t n_chains,
                     uint64_t seed, int64_t step0, float *modes_dev, double *com_dev,
                     int64_t n_steps, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SFP_H */
