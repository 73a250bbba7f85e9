// Kernels for one input kind (depth_f32) except the FD mean's with the error bound
// (tfn_k_depth_f32_fdmean.cu); the instantiations are split by kind so that the
// translation units compile in parallel.
#include "tfn_kernel.cuh"

namespace tfn {
KernelFn kernels_depth_f32(int grad, int phi, int cfg, bool noref)
{
    return dev::select_kernel<KIND_DEPTH_F32, false>(grad, phi, cfg, noref);
}
KernelFn refiners_depth_f32(int grad, int phi) { return dev::select_refiner<KIND_DEPTH_F32>(grad, phi); }
}  // namespace tfn
