// sfp_tc.h -- tensor-core (tcgen05) mode transforms used by the SFP_FP32 path.
#pragma once
#include <cuda_runtime.h>

namespace sfp {

struct TcPlan;

// Record an error message for sfp_last_error() and return `code`.
int report(int code, const char* msg);

// Plan the two transforms of one group with M beads and `rows` = 3 * chains
// state rows: inverse r = phi R (rows rows) and forward [DeltaH|Z] = phi^T [f|z]
// (2 * rows rows).  phi / phiT are the FP64 tables [n][p] / [p][n].
int tc_create(TcPlan** out, int M, int rows, const double* phi, const double* phiT,
              cudaStream_t stream);
// which = 0: inverse, 1: forward.  FP32 in and out, row-major [row][M].
int tc_transform(TcPlan* plan, int which, const float* in, float* out, cudaStream_t stream);
void tc_destroy(TcPlan* plan);

}  // namespace sfp
