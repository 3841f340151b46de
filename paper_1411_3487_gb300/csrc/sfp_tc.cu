// sfp_tc.cu -- placeholder until the tcgen05 transforms land.
#include "../../include/sfp.h"
#include "sfp_tc.h"

namespace sfp {
struct TcPlan { int dummy; };
int tc_create(TcPlan** out, int, int, const double*, const double*, cudaStream_t)
{
    *out = nullptr;
    return report(SFP_ENOTSUP, "tensor-core transforms are not built yet; use SFP_FP32_SIMT");
}
int tc_transform(TcPlan*, int, const float*, float*, cudaStream_t) { return report(SFP_ENOTSUP, "no plan"); }
void tc_destroy(TcPlan*) {}
}  // namespace sfp
