// Radius-4 (8th-order) instantiations of the tensor-memory 3-D step kernel.
#include "k_step3d_tm.cuh"

namespace fwi {

Step3dKernelInfo step3d_kernel_tm4(int mode, bool iso, bool tile_g, bool half)
{
    if (iso) return s3tm::kernel_info<4, s3tm::kPackX | s3tm::kIso>(mode, tile_g, half);
    return s3tm::kernel_info<4, s3tm::kPackX>(mode, tile_g, half);
}

}  // namespace fwi
