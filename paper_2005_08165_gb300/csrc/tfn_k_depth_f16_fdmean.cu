// The FD mean's kernels with the error bound for one input kind (depth_f16), in a
// translation unit of their own (see select_kernel).
#include "tfn_kernel.cuh"

namespace tfn {
KernelFn kernels_depth_f16_fdmean(int cfg)
{
    return dev::select_kernel<KIND_DEPTH_F16, true>(GRAD_FD, PHI_MEAN, cfg, false);
}
}  // namespace tfn
