// The FD mean's kernels with the error bound for one input kind (disp_f32), in a
// translation unit of their own (see select_kernel).
#include "tfn_kernel.cuh"

namespace tfn {
KernelFn kernels_disp_f32_fdmean(int cfg)
{
    return dev::select_kernel<KIND_DISP_F32, true>(GRAD_FD, PHI_MEAN, cfg, false);
}
}  // namespace tfn
