// lbm_kernels.cu -- storage dispatch, launch-configuration names and the final stage of the
// FP64 diagnostics reduction.
#include "lbm_device.cuh"

namespace lbm {

const Launchers& launchers(int storage)
{
    switch (storage) {
    case LBM_STORE_FP32: return launchers_fp32();
    case LBM_STORE_FP16: return launchers_fp16();
    default: return launchers_bf16();
    }
}

const char* launch_config_name(int config)
{
    static const char* names[N_LAUNCH_CONFIGS] = {"256x3", "128x7", "128x6", "128x8", "128x10", "pipe128x6",
                                                            "2c128x4", "2c128x3"};
    return (config >= 0 && config < N_LAUNCH_CONFIGS) ? names[config] : "?";
}

int64_t diagnostics_blocks(int64_t n_fluid)
{
    return n_fluid == 0 ? 1 : (n_fluid + dev::DIAG_THREADS - 1) / dev::DIAG_THREADS;
}

namespace {
__global__ void __launch_bounds__(dev::DIAG_THREADS)
    k_diagnostics_final(const double* partials, int64_t n_blocks, lbm_diagnostics* out)
{
    __shared__ double sh[(dev::DIAG_THREADS / 32) * dev::DIAG_FIELDS];
    double x[dev::DIAG_FIELDS] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t b = threadIdx.x; b < n_blocks; b += dev::DIAG_THREADS)
        for (int f = 0; f < dev::DIAG_FIELDS; ++f) {
            const double p = partials[b * dev::DIAG_FIELDS + f];
            x[f] = (f == 3) ? fmax(x[f], p) : x[f] + p;
        }
    dev::block_reduce5(x, sh);
    if (threadIdx.x == 0) {
        out->mass = x[0];
        out->flux_in = x[1];
        out->flux_out = x[2];
        out->max_u = x[3];
        out->n_nonfinite = (int64_t)x[4];
    }
}
}  // namespace

cudaError_t launch_diagnostics_final(const double* partials, int64_t n_blocks, lbm_diagnostics* out,
                                     cudaStream_t stream)
{
    k_diagnostics_final<<<1, dev::DIAG_THREADS, 0, stream>>>(partials, n_blocks, out);
    return cudaGetLastError();
}

}  // namespace lbm
