// march8_view.cu -- the single-view raymarch kernels with 8 view steps per
// warp iteration (see march_kernels.cuh); each kernel family has its own
// translation unit so that they compile in parallel.
#include "march_kernels.cuh"

namespace cloudvol {
template void launch_march_ch<8>(const SceneParams &, const ViewParams &, const cloud_volume *,
                                  unsigned long long *, int, cudaStream_t);
}  // namespace cloudvol
