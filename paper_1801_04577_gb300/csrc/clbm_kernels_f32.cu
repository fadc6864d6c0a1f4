// FP32 storage, FP32 collision.
#include "clbm_kernels.cuh"

namespace clbm {

const Launchers kLaunchF32 = LaunchImpl<float>::table();

}  // namespace clbm
