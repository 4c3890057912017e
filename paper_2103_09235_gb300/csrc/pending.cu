// Entry points whose kernels are not built yet report STENCIL_ERR_UNSUPPORTED.
#include "plan.h"

namespace sg {

stencil_status_t autotune2d(stencil_plan_s *p, cudaStream_t)
{
    p->tuned_m = 1;
    p->tuned_b = 1;
    p->tuned_ty = 0;
    return STENCIL_OK;
}

}  // namespace sg

extern "C" stencil_status_t stencil_run_batched(int, const stencil_plan_t *, const void *const *,
                                                void *const *, const int64_t *, const int *,
                                                stencil_stream_t)
{
    sg::set_error("batched runs are not built yet");
    return STENCIL_ERR_UNSUPPORTED;
}
