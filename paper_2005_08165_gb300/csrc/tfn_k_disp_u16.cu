// Kernels for one input kind (disp_u16) except the FD mean's with the error bound
// (tfn_k_disp_u16_fdmean.cu); the instantiations are split by kind so that the
// translation units compile in parallel.
#include "tfn_kernel.cuh"

namespace tfn {
KernelFn kernels_disp_u16(int grad, int phi, int cfg, bool noref)
{
    return dev::select_kernel<KIND_DISP_U16, false>(grad, phi, cfg, noref);
}
KernelFn refiners_disp_u16(int grad, int phi) { return dev::select_refiner<KIND_DISP_U16>(grad, phi); }
}  // namespace tfn
