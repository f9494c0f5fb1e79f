// lbm_noalloc.cu -- lbm_get_diagnostics_noalloc: the FP64 diagnostics reduction of a domain
// with its scratch in a fixed device array of this library instead of memory obtained from an
// allocator.
//
// Who needs it: code that must not allocate device memory at the moment it asks for the
// diagnostics -- a monitoring thread in a real-time or latency-bound loop (cudaMalloc can block
// and synchronise the device), or a host application whose device memory is reserved in full by
// another framework's pool, so that a late allocation would fail.  The domain itself is still
// created (and allocated) beforehand; this call only reads it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbm_internal.h"

namespace {

// Scratch of the reduction: per-block partial sums (5 doubles per 256 fluid cells) followed by
// the result record.  Every call shares it, and it keeps the last call's contents; the
// reduction overwrites every word it reads, so nothing has to be cleared between calls.  Two
// calls whose work overlaps on the GPU (domains on different streams, or different host
// threads) race on it.
constexpr int64_t kMaxBlocks = 8192;                                   // 2,097,152 fluid cells
constexpr int64_t kMaxFluid = kMaxBlocks * 256;
constexpr size_t kPartialBytes = sizeof(double) * 5 * (size_t)kMaxBlocks;  // 320 KiB
constexpr size_t kScratchBytes = kPartialBytes + 256;

static __device__ __align__(256) unsigned char g_diag_scratch[kScratchBytes];

// Device address of g_diag_scratch on each device, looked up once per device (with that device
// current).  In host code the symbol is only a host-side stand-in, so the kernels receive this
// looked-up address.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

void err(const std::string& msg) { lbm::set_last_error(msg.c_str()); }

}  // namespace

extern "C" lbm_status lbm_get_diagnostics_noalloc(lbm_domain* dom, lbm_diagnostics* out)
{
    using namespace lbm;
    if (!dom || !out) {
        err("NULL argument");
        return LBM_ERR_INVALID_ARG;
    }
    DomainAccess A;
    if (!domain_access(dom, &A)) {
        err("domain not usable");
        return LBM_ERR_STATE;
    }
    if (A.n_fluid > kMaxFluid) {
        err("lbm_get_diagnostics_noalloc: the domain has " + std::to_string(A.n_fluid) +
                       " fluid cells; its fixed scratch covers at most " + std::to_string(kMaxFluid));
        return LBM_ERR_INVALID_ARG;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess || device < 0 || device >= kMaxDevices) {
        err(std::string("lbm_get_diagnostics_noalloc: no usable current device: ") +
                       cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[device]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_diag_scratch);
            if (e != cudaSuccess) {
                err(std::string("lbm_get_diagnostics_noalloc: cudaGetSymbolAddress failed: ") +
                               cudaGetErrorString(e));
                return LBM_ERR_CUDA;
            }
            g_scratch_ptr[device] = p;
        }
        scratch = g_scratch_ptr[device];
    }
    double* partials = static_cast<double*>(scratch);
    lbm_diagnostics* d_out = reinterpret_cast<lbm_diagnostics*>(static_cast<unsigned char*>(scratch) + kPartialBytes);
    e = launchers(A.storage).diagnostics(A.scheme, *A.view, A.src, A.args, A.fl_slot, A.n_fluid, partials, A.stream);
    if (e == cudaSuccess) e = launch_diagnostics_final(partials, diagnostics_blocks(A.n_fluid), d_out, A.stream);
    lbm_diagnostics h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_out, sizeof(h), cudaMemcpyDeviceToHost, A.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(A.stream);
    if (e != cudaSuccess) {
        err(std::string("lbm_get_diagnostics_noalloc: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    h.time = A.time;
    *out = h;
    if (h.n_nonfinite > 0) {
        err("non-finite populations in " + std::to_string(h.n_nonfinite) + " cells");
        return LBM_ERR_UNSTABLE;
    }
    err("");
    return LBM_OK;
}
