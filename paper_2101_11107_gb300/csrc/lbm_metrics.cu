// lbm_metrics.cu -- the flow metrics of the paper's comparisons on the device: the similarity
// index of two velocity fields (Sec. 3.4) and the output of running means (Sec. 3.3); the
// C-ABI entry point lbm_similarity_index.  The running-mean accumulation and the point probes
// gather populations and live with the other storage-templated kernels (lbm_device.cuh).
//
// The similarity index is a reduction over up to ~10^8 points, bound by reading 6 floats and a
// mask byte per point: grid-stride CTAs, FP64 terms, and fixed-order two-stage reductions (per
// CTA, then one CTA over the CTA partials), so the result is reproducible run to run.  Its
// scratch is a fixed static __device__ array (no allocation); calls are serialised by a mutex.
#include <cmath>
#include <mutex>
#include <string>

#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr int SI_BLOCKS = 608;  // 4 x 152 SMs
constexpr int SI_THREADS = 256;

__device__ double g_si_max[2 * SI_BLOCKS];  // per CTA: max |u_a|, max |u_b|
__device__ double g_si_sum[2 * SI_BLOCKS];  // per CTA: sum of terms, number of points
__device__ double g_si_out;

__device__ __forceinline__ double mag(const float* u, int64_t n, int64_t p)
{
    const double x = u[p], y = u[n + p], z = u[2 * n + p];
    return sqrt(x * x + y * y + z * z);
}

// fixed-order tree reduction of SI_THREADS values in shared memory (op = max or sum)
template <bool MAX>
__device__ double block_reduce(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = SI_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = MAX ? fmax(sh[threadIdx.x], sh[threadIdx.x + s]) : sh[threadIdx.x] + sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SI_THREADS) k_si_max(const float* ua, const float* ub, const uint8_t* mask, int64_t n)
{
    __shared__ double sh[SI_THREADS];
    double ma = 0.0, mb = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * SI_THREADS + threadIdx.x; p < n; p += (int64_t)SI_BLOCKS * SI_THREADS)
        if (!mask || mask[p]) {
            ma = fmax(ma, mag(ua, n, p));
            mb = fmax(mb, mag(ub, n, p));
        }
    ma = block_reduce<true>(ma, sh);
    mb = block_reduce<true>(mb, sh);
    if (threadIdx.x == 0) {
        g_si_max[2 * blockIdx.x] = ma;
        g_si_max[2 * blockIdx.x + 1] = mb;
    }
}

__global__ void __launch_bounds__(SI_THREADS) k_si_sum(const float* ua, const float* ub, const uint8_t* mask, int64_t n)
{
    __shared__ double sh[SI_THREADS];
    double ma = 0.0, mb = 0.0;
    for (int b = threadIdx.x; b < SI_BLOCKS; b += SI_THREADS) {
        ma = fmax(ma, g_si_max[2 * b]);
        mb = fmax(mb, g_si_max[2 * b + 1]);
    }
    ma = block_reduce<true>(ma, sh);
    mb = block_reduce<true>(mb, sh);
    const double ia = ma > 0.0 ? 1.0 / ma : 0.0, ib = mb > 0.0 ? 1.0 / mb : 0.0;
    double sum = 0.0, cnt = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * SI_THREADS + threadIdx.x; p < n; p += (int64_t)SI_BLOCKS * SI_THREADS)
        if (!mask || mask[p]) {
            const double ax = ua[p], ay = ua[n + p], az = ua[2 * n + p];
            const double bx = ub[p], by = ub[n + p], bz = ub[2 * n + p];
            const double na = sqrt(ax * ax + ay * ay + az * az), nb = sqrt(bx * bx + by * by + bz * bz);
            const double cosv = (na > 0.0 && nb > 0.0) ? (ax * bx + ay * by + az * bz) / (na * nb) : 0.0;
            sum += 0.5 * (1.0 + cosv) * (1.0 - fabs(na * ia - nb * ib));
            cnt += 1.0;
        }
    sum = block_reduce<false>(sum, sh);
    cnt = block_reduce<false>(cnt, sh);
    if (threadIdx.x == 0) {
        g_si_sum[2 * blockIdx.x] = sum;
        g_si_sum[2 * blockIdx.x + 1] = cnt;
    }
}

__global__ void __launch_bounds__(SI_THREADS) k_si_final()
{
    __shared__ double sh[SI_THREADS];
    double sum = 0.0, cnt = 0.0;
    for (int b = threadIdx.x; b < SI_BLOCKS; b += SI_THREADS) {
        sum += g_si_sum[2 * b];
        cnt += g_si_sum[2 * b + 1];
    }
    sum = block_reduce<false>(sum, sh);
    cnt = block_reduce<false>(cnt, sh);
    if (threadIdx.x == 0) g_si_out = cnt > 0.0 ? sum / cnt : 0.0;
}

__global__ void __launch_bounds__(256) k_mean_out(const Sum4* sums, const int32_t* fl_box, int64_t n_fluid,
                                                  double inv, int dense, float* rho, float* u, int64_t n_out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_fluid) return;
    const Sum4 s = sums[k];
    const int64_t o = dense ? (int64_t)fl_box[k] : k;
    rho[o] = (float)(s.x * inv);
    u[o] = (float)(s.y * inv);
    u[n_out + o] = (float)(s.z * inv);
    u[2 * n_out + o] = (float)(s.w * inv);
}

std::mutex g_si_mutex;

lbm_status si_fail(lbm_status s, const std::string& msg)
{
    set_last_error(msg.c_str());
    return s;
}

}  // namespace

namespace lbm {

cudaError_t launch_mean_out(const Sum4* sums, const int32_t* fl_box, int64_t n_fluid, int64_t n_samples, int dense,
                            float* rho, float* u, int64_t n_out, cudaStream_t stream)
{
    if (n_fluid == 0) return cudaSuccess;
    const int grid = (int)((n_fluid + 255) / 256);
    k_mean_out<<<grid, 256, 0, stream>>>(sums, fl_box, n_fluid, 1.0 / (double)n_samples, dense, rho, u, n_out);
    return cudaGetLastError();
}

}  // namespace lbm

extern "C" lbm_status lbm_similarity_index(const float* u_a, const float* u_b, const uint8_t* mask, int64_t n,
                                           double* si, void* cuda_stream)
{
    set_last_error("");
    if (!u_a || !u_b || !si || n < 0) return si_fail(LBM_ERR_INVALID_ARG, "NULL argument or negative size");
    std::lock_guard<std::mutex> lock(g_si_mutex);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_si_max<<<SI_BLOCKS, SI_THREADS, 0, s>>>(u_a, u_b, mask, n);
    k_si_sum<<<SI_BLOCKS, SI_THREADS, 0, s>>>(u_a, u_b, mask, n);
    k_si_final<<<1, SI_THREADS, 0, s>>>();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(si, g_si_out, sizeof(double), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return si_fail(LBM_ERR_CUDA, std::string("similarity index: ") + cudaGetErrorString(e));
    return LBM_OK;
}
