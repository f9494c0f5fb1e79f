// lbm_step_fp32.cu -- kernels and launchers of the FP32 population storage (see lbm_device.cuh).
#include "lbm_device.cuh"

namespace lbm {
const Launchers& launchers_fp32() { return dev::make_launchers<LBM_STORE_FP32>(); }
}  // namespace lbm
