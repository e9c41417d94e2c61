// Radius-8 (16th-order) instantiations of the TMA-staged 3-D step kernel.
#include "k_step3d.cuh"

namespace fwi {

namespace {
template <int TY, int RY, int P>
Step3dKernelInfo info(int mode)
{
    using C = s3d::Cfg<8, TY, RY, P>;
    Step3dKernelInfo k;
    k.fn = mode == kModeStep ? (Step3dKernel)s3d::k_step3d_tma<8, TY, RY, P, kModeStep>
                             : (Step3dKernel)s3d::k_step3d_tma<8, TY, RY, P, kModeImage>;
    k.threads = C::NT;
    k.smem = C::SMEM;
    return k;
}
}  // namespace

Step3dKernelInfo step3d_kernel_m8(const Step3dVariant &v, int mode)
{
    if (v.unroll) return Step3dKernelInfo{nullptr, 0, 0};
    if (v.ty == 32 && v.ry == 2 && v.pf == 2) return info<32, 2, 2>(mode);
    if (v.ty == 32 && v.ry == 1 && v.pf == 2) return info<32, 1, 2>(mode);
    if (v.ty == 24 && v.ry == 2 && v.pf == 3) return info<24, 2, 3>(mode);
    if (v.ty == 24 && v.ry == 1 && v.pf == 3) return info<24, 1, 3>(mode);
    if (v.ty == 16 && v.ry == 1 && v.pf == 4) return info<16, 1, 4>(mode);
    return Step3dKernelInfo{nullptr, 0, 0};
}

}  // namespace fwi
