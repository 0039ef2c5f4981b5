// Tensor-core M2L (placeholder until the tcgen05 kernel lands).
#include "common.cuh"
#include "vfmm_internal.h"

namespace vfmm {

int launch_split(Ctx *c, int, bool)
{
    c->last_error = "tensor-core M2L not built";
    return VFMM_ERR_UNSUPPORTED;
}

int launch_tc_m2l(Ctx *c, int, const int4 *, const int *, const int *, bool)
{
    c->last_error = "tensor-core M2L not built";
    return VFMM_ERR_UNSUPPORTED;
}

}  // namespace vfmm
