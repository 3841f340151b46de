// sfp_internal.h -- slot-level access to a batch for the serving loop
// (sfp_server.cu).  A serving pool is a batch of one length group whose chains
// are slots: each slot carries its own job key, step counter and stop step.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/sfp.h"

namespace sfp {

// Stop every slot (stop step 0): nothing advances until a slot is started.
int internal_idle_all(sfp_batch* b);
// Start n slots: equilibrium start keyed by (seed, jobs[i]) (Philox counter
// (0, 0, k, 1)), centre of mass at the origin, step counter 0, stop step
// stops[i], shear rate shear_per_s[i] (1/s).  Asynchronous on the batch stream.
int internal_slots_start(sfp_batch* b, const int32_t* slots, const uint32_t* jobs, const int64_t* stops,
                         const double* shear_per_s, int32_t n);
// Read n slots: modes[i][3][M] (FP64, scaled units, R_0 = sqrt(M) r_cm), centre of
// mass in nm [i][3], step counters; any pointer may be NULL.  Synchronous on
// `stream` (NULL: the batch's stream), after `after` (NULL: no wait).  Stopped
// slots do not change, so a read on another stream may run beside later steps.
int internal_slots_read(sfp_batch* b, const int32_t* slots, int32_t n, double* modes, double* com_nm,
                        int64_t* steps, cudaStream_t stream = nullptr, cudaEvent_t after = nullptr);
// The fused step of the pool covers slots [0, n) only (n < 0: all): the
// slots past the highest running one hold no running job.  Host only.
int internal_set_active(sfp_batch* b, int64_t n);
// Beads, step, slot count and device bytes of a pool.
int internal_shape(const sfp_batch* b, int32_t* M, double* dtau, int32_t* C, size_t* bytes);

}  // namespace sfp
