// lbm_step_bf16.cu -- kernels and launchers of the BF16 population storage (see lbm_device.cuh).
#include "lbm_device.cuh"

namespace lbm {
const Launchers& launchers_bf16() { return dev::make_launchers<LBM_STORE_BF16>(); }
}  // namespace lbm
