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

namespace {
// One thread per face position; every value is copied as raw bits (storage precision), so the
// exchange is exact.
template <typename T, bool PACK>
__global__ void __launch_bounds__(256)
    k_halo_copy(T* __restrict__ pop, uint32_t n_slots, const int32_t* __restrict__ slot, int64_t area, HaloDirs dirs,
                T* __restrict__ buf)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= area) return;
    const int32_t s = slot[p];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const uint32_t off = (uint32_t)dirs.d[j] * n_slots + (uint32_t)s;
        if (PACK) buf[j * area + p] = s >= 0 ? pop[off] : T(0);
        else if (s >= 0) pop[off] = buf[j * area + p];
    }
}
}  // namespace

cudaError_t launch_halo_copy(int bytes_per_value, bool pack, void* pop, int64_t n_slots, const int32_t* slot,
                             int64_t area, const HaloDirs& dirs, void* buf, cudaStream_t stream)
{
    if (area == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((area + 255) / 256);
    if (bytes_per_value == 4) {
        if (pack)
            k_halo_copy<uint32_t, true><<<grid, 256, 0, stream>>>(static_cast<uint32_t*>(pop), (uint32_t)n_slots, slot,
                                                                 area, dirs, static_cast<uint32_t*>(buf));
        else
            k_halo_copy<uint32_t, false><<<grid, 256, 0, stream>>>(static_cast<uint32_t*>(pop), (uint32_t)n_slots, slot,
                                                                  area, dirs, static_cast<uint32_t*>(buf));
    } else {
        if (pack)
            k_halo_copy<uint16_t, true><<<grid, 256, 0, stream>>>(static_cast<uint16_t*>(pop), (uint32_t)n_slots, slot,
                                                                 area, dirs, static_cast<uint16_t*>(buf));
        else
            k_halo_copy<uint16_t, false><<<grid, 256, 0, stream>>>(static_cast<uint16_t*>(pop), (uint32_t)n_slots, slot,
                                                                  area, dirs, static_cast<uint16_t*>(buf));
    }
    return cudaGetLastError();
}

cudaError_t launch_diagnostics_final(const double* partials, int64_t n_blocks, lbm_diagnostics* out,
                                     cudaStream_t stream)
{
    k_diagnostics_final<<<1, dev::DIAG_THREADS, 0, stream>>>(partials, n_blocks, out);
    return cudaGetLastError();
}

}  // namespace lbm
