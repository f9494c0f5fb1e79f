// lbm_step_fp16.cu -- kernels and launchers of the FP16 population storage (see lbm_device.cuh).
#include "lbm_device.cuh"

namespace lbm {
const Launchers& launchers_fp16() { return dev::make_launchers<LBM_STORE_FP16>(); }
}  // namespace lbm
