// The FD mean's kernels with the error bound for one input kind (disp_u16), in a
// translation unit of their own (see select_kernel).
#include "tfn_kernel.cuh"

namespace tfn {
KernelFn kernels_disp_u16_fdmean(int cfg)
{
    return dev::select_kernel<KIND_DISP_U16, true>(GRAD_FD, PHI_MEAN, cfg, false);
}
}  // namespace tfn
