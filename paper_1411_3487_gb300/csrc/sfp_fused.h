// sfp_fused.h -- the fused mode-space step (one kernel per step and length
// group) of the SFP_FP32 path.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sfp {

struct FusedPlan;

// Device pointers and scalars of one length group, read by every launch.
struct FusedArgs {
    float* R;               // [C][3][M] mode amplitudes, p = 0 slots held at 0
    double* com;            // [C][3] centre of mass (scaled units)
    int64_t* step;          // [C] Philox step counters
    const int64_t* stop;    // [C] a chain advances only while step < stop (NULL: no limit)
    const uint32_t* job;    // [C] Philox key word 1
    const double* shear;    // [C] shear rate in 1/tau
    const float* dm;        // [M] 1 - e^{-zeta_p dtau}
    const float* g;         // [M] shear weights (g_0 = dtau)
    int* err;               // bit 0: non-finite state, bit 1: a pipeline wait timed out,
                            // bit 2: a 512-bead step launched without its cluster of two
    int C;
    float c12nu;            // 1 - 2 nu
    uint32_t seed;
    double inv_sqrtM;
    double dtau;
    int n_steps;            // steps per launch (>= 1)
    int cpt;                // chains per tile (4..40, a multiple of 4), as in the plan (fused_tile)
    int stall_test;         // 1: the MMA thread first waits on a barrier nothing arrives at (tests the bounded waits)
    float* zbuf;            // mode-keyed noise: Z of two steps [2][C][3][M] (set by fused_step from the plan)
    const float* w;         // mode-keyed noise: w_p, w_0 of the centre of mass (set by fused_step)
};

// True when a group of M beads can take the fused step (M = 64, 128 or 256).
bool fused_supported(int M);

// Tables of one group: chi [n][p] (row n = 0 and column p = 0 zero), phi [n][p],
// and the per-mode weights h_p (Eq. f2), w_p (Eq. d6; w[0] = sqrt(2 T* dtau)).
// The forward table F = [h_p chi_{n,p} ; w_p phi_{n,p}] (2M rows p, M columns n)
// and chi are split once into TF32 hi / lo.  R is the group's state array.
// bf16: BF16 hi/lo operands (kind::f16) instead of the TF32 split; two (with
// bf16): two passes A_lo B_hi + A_hi B_hi, the tables as their BF16 hi part.
int fused_create(FusedPlan** out, int M, int C, const double* chi, const double* phi, const double* h,
                 const double* w, float* R, cudaStream_t stream, bool bf16 = false, bool two = false);
// args.n_steps steps of every chain of the group, in one launch.
int fused_step(FusedPlan* plan, const FusedArgs& args, cudaStream_t stream);
// Chains per tile of the plan, and a new value (1..40, rounded up to a multiple
// of 4: one share per TMEM lane quarter; rebuilds the R map).
int fused_tile(const FusedPlan* plan);
// CTAs that run one tile: 2 at M = 512 (a cluster pair), else 1.
int fused_ctas_per_tile(const FusedPlan* plan);
// Device bytes the plan's tables hold.
size_t fused_bytes(const FusedPlan* plan);
int fused_set_tile(FusedPlan* plan, int cpt);
// Mode-keyed noise on (Z drawn per mode, Eq. c4 reading; M <= 256 only: the
// 512-bead cluster kernel draws bead noise): allocates the plan's Z buffer.
int fused_set_mode_noise(FusedPlan* plan, bool on);
bool fused_mode_noise_supported(int M);
// True for plans that the grouped launch takes (every fused plan).
bool fused_groupable(const FusedPlan* plan);
// One launch of clusters of two CTAs for up to four plans of different lengths
// (64, 128, 256, 512) and the same arithmetic, with the args each would get
// from fused_step (the same n_steps): the 512-bead tiles first (a cluster
// each), then the others two per cluster, longest first.  Same trajectories as
// one fused_step per plan.
int fused_step_grouped(FusedPlan* const* plans, const FusedArgs* args, int n, cudaStream_t stream);
void fused_destroy(FusedPlan* plan);

}  // namespace sfp
