// Radius-4 (8th-order) instantiations of the TMA-staged 3-D step kernel.
#include "k_step3d.cuh"

namespace fwi {

Step3dKernelInfo step3d_kernel_m4(const Step3dVariant &v, int mode, bool iso)
{
    if (v.tm) return step3d_kernel_tm4(mode, iso, v.tile_g != 0, v.half != 0);
    const int opt = mode == kModeStep ? v.opt : v.opt_rev;
    if (iso && v.ty == 16 && v.ry == 2 && v.pf == 3 && v.u == 2 && opt == 0)
        return s3d::kernel_info<4, 16, 2, 3, 2, s3d::kIso>(mode);
    if (v.ty == 16 && v.ry == 2 && v.pf == 3) {
        if (v.u == 2 && opt == 0) return s3d::kernel_info<4, 16, 2, 3, 2, 0>(mode);
        if (v.u == 1 && opt == 0) return s3d::kernel_info<4, 16, 2, 3, 1, 0>(mode);
    }
    return Step3dKernelInfo{nullptr, 0, 0};
}

}  // namespace fwi
