// march16_view.cu -- the single-view raymarch kernels with 16 view steps per
// warp iteration (see march_kernels.cuh); each kernel family has its own
// translation unit so that they compile in parallel.
#include "march_kernels.cuh"

namespace cloudvol {
template void launch_march_ch<16>(const SceneParams &, const ViewParams &, const cloud_volume *,
                                  unsigned long long *, int, cudaStream_t);
}  // namespace cloudvol
