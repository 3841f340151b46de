// sfp_tc.h -- tensor-core (tcgen05) mode transforms used by the SFP_FP32 path.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace sfp {

struct TcPlan;

// Record an error message for sfp_last_error() and return `code`.
int report(int code, const char* msg);

// True when a group of M beads can use the tensor-core transforms
// (M = 32, 64, 128, 256 or 512; other lengths keep the CUDA-core transforms).
bool tc_supported(int M);

// Plan the two transforms of one group with M beads and `rows` = 3 * chains:
// inverse u = chi R (bond vectors, Eq. e5) reads R [rows][M] and writes r_out;
// forward DeltaH = chi^T v (Eq. e11) and Z = phi^T z (Eq. c4) read
// fz = [v | z] [2 rows][M] and write yz_out = [DeltaH | Z].
// chi [n][p], chiT [p][n] and phiT [p][n] are FP64 tables; they are split
// once into TF32 (or, with bf16, BF16) hi / lo parts; two (with bf16): two
// passes A_lo B_hi + A_hi B_hi, the tables as their BF16 hi part alone.
// A wait that times out inside the kernel sets bit 2 of *err.
int tc_create(TcPlan** out, int M, int rows, const double* chi, const double* chiT, const double* phiT,
              const float* R, float* r_out, const float* fz, float* yz_out, int* err, cudaStream_t stream,
              bool bf16 = false, bool two = false);
// which: 0 inverse (u = chi R), 1 forward (DeltaH = chi^T v and Z = phi^T z), 2 the forward force half alone.
int tc_transform(TcPlan* plan, int which, cudaStream_t stream);
// Device bytes the plan's tables hold.
size_t tc_bytes(const TcPlan* plan);
void tc_destroy(TcPlan* plan);

}  // namespace sfp
