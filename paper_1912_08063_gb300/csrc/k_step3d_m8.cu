// Radius-8 (16th-order) instantiations of the TMA-staged 3-D step kernel.
#include "k_step3d.cuh"

namespace fwi {

Step3dKernelInfo step3d_kernel_m8(const Step3dVariant &v, int mode)
{
    if (v.ty == 32 && v.ry == 2 && v.pf == 2 && v.opt == 0) {
        if (v.u == 3) return s3d::kernel_info<8, 32, 2, 2, 3, 0>(mode);
        if (v.u == 1) return s3d::kernel_info<8, 32, 2, 2, 1, 0>(mode);
    }
    if (v.ty == 32 && v.ry == 1 && v.pf == 2 && v.opt == 0) {
        if (v.u == 2) return s3d::kernel_info<8, 32, 1, 2, 2, 0>(mode);
        if (v.u == 3) return s3d::kernel_info<8, 32, 1, 2, 3, 0>(mode);
        if (v.u == 4) return s3d::kernel_info<8, 32, 1, 2, 4, 0>(mode);
    }
    return Step3dKernelInfo{nullptr, 0, 0};
}

}  // namespace fwi
