// IEEE binary16 deviation storage, FP32 collision.
#include "clbm_kernels.cuh"

namespace clbm {

const Launchers kLaunchF16 = LaunchImpl<__half>::table();

}  // namespace clbm
