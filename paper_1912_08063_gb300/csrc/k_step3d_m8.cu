// Radius-8 (16th-order) instantiations of the TMA-staged 3-D step kernel.
#include "k_step3d.cuh"

namespace fwi {

Step3dKernelInfo step3d_kernel_m8(const Step3dVariant &v, int mode, bool iso)
{
    if (v.tm) return step3d_kernel_tm8(mode, iso, v.tile_g != 0, v.half != 0);
    const int opt = mode == kModeStep ? v.opt : v.opt_rev;
    if (iso && v.ty == 32 && v.ry == 2 && v.pf == 2 && v.u == 2 && opt == 1)
        return s3d::kernel_info<8, 32, 2, 2, 2, 1 | s3d::kIso>(mode);
    if (v.ty == 32 && v.ry == 2 && v.pf == 2) {
        if (v.u == 2 && opt == 1) return s3d::kernel_info<8, 32, 2, 2, 2, 1>(mode);
        if (v.u == 2 && opt == 0) return s3d::kernel_info<8, 32, 2, 2, 2, 0>(mode);
        if (v.u == 3 && opt == 0) return s3d::kernel_info<8, 32, 2, 2, 3, 0>(mode);
    }
    return Step3dKernelInfo{nullptr, 0, 0};
}

}  // namespace fwi
