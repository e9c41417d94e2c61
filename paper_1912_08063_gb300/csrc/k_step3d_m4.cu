// Radius-4 (8th-order) instantiations of the TMA-staged 3-D step kernel.
#include "k_step3d.cuh"

namespace fwi {

namespace {
template <int TY, int RY, int P, bool UNR>
Step3dKernelInfo info(int mode)
{
    using C = s3d::Cfg<4, TY, RY, P>;
    Step3dKernelInfo k;
    k.fn = mode == kModeStep ? (Step3dKernel)s3d::k_step3d_tma<4, TY, RY, P, kModeStep, UNR>
                             : (Step3dKernel)s3d::k_step3d_tma<4, TY, RY, P, kModeImage, UNR>;
    k.threads = C::NT;
    k.smem = C::SMEM;
    return k;
}
}  // namespace

Step3dKernelInfo step3d_kernel_m4(const Step3dVariant &v, int mode)
{
    if (v.ty == 16 && v.ry == 1 && v.pf == 3 && v.unroll) return info<16, 1, 3, true>(mode);
    if (v.ty == 16 && v.ry == 1 && v.pf == 3 && !v.unroll) return info<16, 1, 3, false>(mode);
    if (v.ty == 16 && v.ry == 2 && v.pf == 3 && v.unroll) return info<16, 2, 3, true>(mode);
    if (v.ty == 16 && v.ry == 2 && v.pf == 3 && !v.unroll) return info<16, 2, 3, false>(mode);
    return Step3dKernelInfo{nullptr, 0, 0};
}

}  // namespace fwi
