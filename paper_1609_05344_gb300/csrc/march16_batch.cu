// march16_batch.cu -- the persistent multi-view raymarch kernels with 16 view
// steps per warp iteration (see march_kernels.cuh).
#include "march_kernels.cuh"

namespace cloudvol {
template const void *batch_kernel_ch<16>(int, int, bool, int);
}  // namespace cloudvol
