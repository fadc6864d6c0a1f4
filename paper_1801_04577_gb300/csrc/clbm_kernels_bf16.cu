// bfloat16 deviation storage, FP32 collision.
#include "clbm_kernels.cuh"

namespace clbm {

const Launchers kLaunchBF16 = LaunchImpl<__nv_bfloat16>::table();

}  // namespace clbm
