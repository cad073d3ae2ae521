// march8_batch.cu -- the persistent multi-view raymarch kernels with 8 view
// steps per warp iteration (see march_kernels.cuh).
#include "march_kernels.cuh"

namespace cloudvol {
template const void *batch_kernel_ch<8>(int, int, bool, int);
}  // namespace cloudvol
