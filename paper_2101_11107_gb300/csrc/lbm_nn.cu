// lbm_nn.cu -- the learned coarse-grid corrector: a 3-layer 3-D convolutional network
// (16 channels, 3x3x3 kernels, BF16 weights and activations, FP32 accumulation), its backward
// pass and Adam training, the restriction of fine fields onto the coarse grid, and the C-ABI
// entry points lbm_corrector_* / lbm_restrict.
//
// The paper has no learned component; its Sec. 3.4 shows that a 2x coarser grid keeps useful
// accuracy at ~14x less cost.  The corrector nudges the coarse velocity toward the fine solution
// restricted onto the coarse grid, every K coarse steps.
//
// GB300 design:
//   * Activations are channels-last BF16 on the coarse box padded by one zero cell on every side
//     (16 channels = 32 B per cell), so a 3x3x3 neighbourhood never needs a bounds test.
//   * Only 4^3 tiles that hold fluid, dilated by one tile, are evaluated (the rest of the box
//     stays zero): the receptive field of the three layers is 3 cells, so outputs at fluid cells
//     equal those of the dense network.
//   * Convolution = implicit GEMM on the tensor cores with warp-level mma.sync m16n8k16 (BF16 in,
//     FP32 accumulate): a CTA per tile, a warp per 4x4 z-slice (M = 16 cells), N = 16 output
//     channels (two n8 tiles), K = 27 offsets x 16 input channels; the CTA's weights sit in
//     shared memory.  The data-gradient is the same kernel with the flipped, transposed kernel
//     and a ReLU gate; the weight-gradient is a GEMM over cells (M = 16 output channels,
//     N = 16 input channels, K = cells) with per-CTA register accumulation and one FP32 atomic
//     per weight per CTA.
#include <cuda_bf16.h>

#include <cmath>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr int CH = 16;
constexpr int NW = 27 * CH * CH;         // weights per layer
constexpr int NP = 3 * (NW + CH);        // parameters: W1, b1, W2, b2, W3, b3

struct Box {
    int nx, ny, nz;  // interior
    int px, py, pz;  // padded (n + 2)
};

__device__ __forceinline__ size_t pidx(const Box& b, int x, int y, int z)
{
    return ((size_t)(z + 1) * b.py + (size_t)(y + 1)) * b.px + (size_t)(x + 1);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// out[p][co] = act(sum_o sum_ci w[o][co][ci] in[p + o][ci] + bias[co]), zeroed where gate <= 0.
// OUT_F32: write channels 0..3 as FP32 to a dense unpadded [cells][4] array; else BF16 padded.
template <bool OUT_F32>
__global__ void __launch_bounds__(128)
    k_conv(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
           int relu, const __nv_bfloat16* __restrict__ gate, void* __restrict__ out, const int4* __restrict__ tiles, Box b)
{
    __shared__ __align__(16) __nv_bfloat16 sw[NW];
    for (int t = threadIdx.x; t < NW / 8; t += blockDim.x)
        reinterpret_cast<uint4*>(sw)[t] = __ldg(reinterpret_cast<const uint4*>(w) + t);
    __syncthreads();
    const int4 tile = tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int z = tile.z + warp;
    const int xa = tile.x + (g & 3), ya = tile.y + (g >> 2);  // A rows g and g + 8
    const int yb = ya + 2;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const uint32_t* in32 = reinterpret_cast<const uint32_t*>(in);
    const uint32_t* sw32 = reinterpret_cast<const uint32_t*>(sw);
#pragma unroll 3
    for (int o = 0; o < 27; ++o) {
        const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
        const size_t ca = pidx(b, xa + dx, ya + dy, z + dz) * CH / 2, cb = pidx(b, xa + dx, yb + dy, z + dz) * CH / 2;
        uint32_t a[4];
        a[0] = __ldg(in32 + ca + t);
        a[1] = __ldg(in32 + cb + t);
        a[2] = __ldg(in32 + ca + t + 4);
        a[3] = __ldg(in32 + cb + t + 4);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            uint32_t bb[2];
            bb[0] = sw32[(o * CH * CH + (8 * j + g) * CH) / 2 + t];
            bb[1] = sw32[(o * CH * CH + (8 * j + g) * CH) / 2 + t + 4];
            mma16816(acc[j], a, bb);
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co = 8 * j + 2 * t;
            const int y = h ? yb : ya;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (bias) {
                v0 += bias[co];
                v1 += bias[co + 1];
            }
            if (relu) {
                v0 = fmaxf(v0, 0.0f);
                v1 = fmaxf(v1, 0.0f);
            }
            const size_t pc = pidx(b, xa, y, z);
            if (gate) {
                if (!(__bfloat162float(gate[pc * CH + co]) > 0.0f)) v0 = 0.0f;
                if (!(__bfloat162float(gate[pc * CH + co + 1]) > 0.0f)) v1 = 0.0f;
            }
            if (OUT_F32) {
                if (co < 4) {
                    float* o4 = static_cast<float*>(out) + (((size_t)z * b.ny + y) * b.nx + xa) * 4;
                    o4[co] = v0;
                    o4[co + 1] = v1;
                }
            } else {
                __nv_bfloat162 v = __floats2bfloat162_rn(v0, v1);
                *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(out) + pc * CH + co) = v;
            }
        }
}

// dW[o][co][ci] += sum_p dy[p][co] x[p + o][ci] and db[co] += sum_p dy[p][co] over the tiles;
// each warp owns offsets warp, warp + 4, ...; one atomic per weight per CTA at the end.
__global__ void __launch_bounds__(128)
    k_wgrad(const __nv_bfloat16* __restrict__ dy, const __nv_bfloat16* __restrict__ x, const int4* __restrict__ tiles,
            int n_tiles, Box b, float* __restrict__ dW, float* __restrict__ db)
{
    __shared__ __align__(16) __nv_bfloat16 sdy[64 * CH];
    __shared__ __align__(16) __nv_bfloat16 sx[216 * CH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float acc[7][2][4];
#pragma unroll
    for (int l = 0; l < 7; ++l)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[l][j][k] = 0.0f;
    float dbacc = 0.0f;
    for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const int4 tile = tiles[ti];
        __syncthreads();
        {
            const int c = threadIdx.x >> 1, half = threadIdx.x & 1;
            const int cx = c & 3, cy = (c >> 2) & 3, cz = c >> 4;
            reinterpret_cast<uint4*>(sdy)[threadIdx.x] = __ldg(
                reinterpret_cast<const uint4*>(dy + pidx(b, tile.x + cx, tile.y + cy, tile.z + cz) * CH) + half);
        }
        for (int q = threadIdx.x; q < 216 * 2; q += blockDim.x) {
            const int c = q >> 1, half = q & 1;
            const int hx = c % 6, hy = (c / 6) % 6, hz = c / 36;
            reinterpret_cast<uint4*>(sx)[q] = __ldg(
                reinterpret_cast<const uint4*>(x + pidx(b, tile.x - 1 + hx, tile.y - 1 + hy, tile.z - 1 + hz) * CH) + half);
        }
        __syncthreads();
        if (threadIdx.x < CH)
            for (int c = 0; c < 64; ++c) dbacc += __bfloat162float(sdy[c * CH + threadIdx.x]);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            // A[m = co][k = cell c of slab z = s] = dy[cell][co]
            const int k0 = s * 16 + 2 * t, k1 = k0 + 8;
            uint32_t a[4];
            a[0] = pack2(sdy[k0 * CH + g], sdy[(k0 + 1) * CH + g]);
            a[1] = pack2(sdy[k0 * CH + g + 8], sdy[(k0 + 1) * CH + g + 8]);
            a[2] = pack2(sdy[k1 * CH + g], sdy[(k1 + 1) * CH + g]);
            a[3] = pack2(sdy[k1 * CH + g + 8], sdy[(k1 + 1) * CH + g + 8]);
#pragma unroll
            for (int l = 0; l < 7; ++l) {
                const int o = warp + 4 * l;
                if (o >= 27) continue;
                const int dx = o % 3 - 1, dyy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                // B[k = cell c][n = ci] = x[cell(c) + o][ci], halo cell of cell c
                auto hidx = [&](int c) {
                    return ((s + 1 + dz) * 6 + ((c >> 2) + 1 + dyy)) * 6 + ((c & 3) + 1 + dx);
                };
                const int h0 = hidx(2 * t), h1 = hidx(2 * t + 1), h2 = hidx(2 * t + 8), h3 = hidx(2 * t + 9);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int n = 8 * j + g;
                    uint32_t bb[2];
                    bb[0] = pack2(sx[h0 * CH + n], sx[h1 * CH + n]);
                    bb[1] = pack2(sx[h2 * CH + n], sx[h3 * CH + n]);
                    mma16816(acc[l][j], a, bb);
                }
            }
        }
    }
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        const int o = warp + 4 * l;
        if (o >= 27) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int ci = 8 * j + 2 * t;
            atomicAdd(&dW[(o * CH + g) * CH + ci], acc[l][j][0]);
            atomicAdd(&dW[(o * CH + g) * CH + ci + 1], acc[l][j][1]);
            atomicAdd(&dW[(o * CH + g + 8) * CH + ci], acc[l][j][2]);
            atomicAdd(&dW[(o * CH + g + 8) * CH + ci + 1], acc[l][j][3]);
        }
    }
    if (threadIdx.x < CH) atomicAdd(&db[threadIdx.x], dbacc);
}

// Input features on the padded box: u / u_scale (3), (rho - 1) / rho_scale, fluid mask, zeros.
__global__ void k_features(const float* __restrict__ rho, const float* __restrict__ u, const uint8_t* __restrict__ mask,
                           Box b, float inv_us, float inv_rs, __nv_bfloat16* __restrict__ x0)
{
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int x = (int)(c % b.nx), y = (int)((c / b.nx) % b.ny), z = (int)(c / ((int64_t)b.nx * b.ny));
    const float fl = mask[c] ? 1.0f : 0.0f;
    __nv_bfloat16 v[CH];
    v[0] = __float2bfloat16_rn(u[c] * inv_us * fl);
    v[1] = __float2bfloat16_rn(u[n + c] * inv_us * fl);
    v[2] = __float2bfloat16_rn(u[2 * n + c] * inv_us * fl);
    v[3] = __float2bfloat16_rn((rho[c] - 1.0f) * inv_rs * fl);
    v[4] = __float2bfloat16_rn(fl);
#pragma unroll
    for (int k = 5; k < CH; ++k) v[k] = __float2bfloat16_rn(0.0f);
    uint4* dst = reinterpret_cast<uint4*>(x0 + pidx(b, x, y, z) * CH);
    dst[0] = *reinterpret_cast<uint4*>(&v[0]);
    dst[1] = *reinterpret_cast<uint4*>(&v[8]);
}

// du = du_scale * clamp(O[0:3], -clip, clip) at fluid cells, 0 elsewhere (three planes).
__global__ void k_output(const float* __restrict__ o4, const uint8_t* __restrict__ mask, int64_t n, float du_scale,
                         float clip, float* __restrict__ du)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const float fl = mask[c] ? du_scale : 0.0f;
    du[c] = fminf(fmaxf(o4[c * 4 + 0], -clip), clip) * fl;
    du[n + c] = fminf(fmaxf(o4[c * 4 + 1], -clip), clip) * fl;
    du[2 * n + c] = fminf(fmaxf(o4[c * 4 + 2], -clip), clip) * fl;
}

// Loss = mean over fluid cells and components of (O - T)^2, T = (u_target - u) / du_scale;
// dO = 2 (O - T) / N at fluid cells (BF16, padded, channels 0..2).
__global__ void k_count(const uint8_t* __restrict__ mask, int64_t n, unsigned long long* __restrict__ count)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned int ballot = __ballot_sync(0xffffffffu, c < n && mask[c] != 0);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(count, (unsigned long long)__popc(ballot));
}

__global__ void k_loss(const float* __restrict__ o4, const float* __restrict__ u, const float* __restrict__ ut,
                       const uint8_t* __restrict__ mask, Box b, float inv_du, const unsigned long long* __restrict__ count,
                       __nv_bfloat16* __restrict__ dO, double* __restrict__ loss)
{
    __shared__ double sh[8];
    const float two_over_n = *count ? 2.0f / (3.0f * (float)*count) : 0.0f;
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (c < n) {
        // zero the output gradient of every cell, so that a mask differing from the previous
        // call's leaves no stale values behind
        const int x = (int)(c % b.nx), y = (int)((c / b.nx) % b.ny), z = (int)(c / ((int64_t)b.nx * b.ny));
        __nv_bfloat16* d = dO + pidx(b, x, y, z) * CH;
        const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
        d[0] = zero;
        d[1] = zero;
        d[2] = zero;
    }
    if (c < n && mask[c]) {
        const int x = (int)(c % b.nx), y = (int)((c / b.nx) % b.ny), z = (int)(c / ((int64_t)b.nx * b.ny));
        __nv_bfloat16* d = dO + pidx(b, x, y, z) * CH;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float r = o4[c * 4 + k] - (ut[k * n + c] - u[k * n + c]) * inv_du;
            part += (double)r * r;
            d[k] = __float2bfloat16_rn(two_over_n * r);
        }
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        atomicAdd(loss, s);
    }
}

// BF16 forward weights and, for layers 2 and 3, the data-gradient kernels
// wt[o'][ci][co] = w[26 - o'][co][ci] (flipped offsets, transposed channels).
__global__ void k_prepare(const float* __restrict__ master, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * NW) return;
    const int l = i / NW, r = i % NW;
    const int o = r / (CH * CH), co = (r / CH) % CH, ci = r % CH;
    const float v = master[l * (NW + CH) + r];
    wb[i] = __float2bfloat16_rn(v);
    wt[l * NW + ((26 - o) * CH + ci) * CH + co] = __float2bfloat16_rn(v);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// coarse (X,Y,Z) = mean of rho and u over the fluid fine children (2X+a, 2Y+b, 2Z+c); 0 if none.
__global__ void k_restrict(const float* __restrict__ frho, const float* __restrict__ fu, const uint8_t* __restrict__ fmask,
                           int fnx, int fny, int fnz, float* __restrict__ crho, float* __restrict__ cu)
{
    const int cnx = fnx / 2, cny = fny / 2, cnz = fnz / 2;
    const int64_t cn = (int64_t)cnx * cny * cnz, fn = (int64_t)fnx * fny * fnz;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cn) return;
    const int X = (int)(c % cnx), Y = (int)((c / cnx) % cny), Z = (int)(c / ((int64_t)cnx * cny));
    float sr = 0.f, su[3] = {0.f, 0.f, 0.f};
    int k = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int64_t f = (int64_t)(2 * X + dx) + (int64_t)fnx * ((2 * Y + dy) + (int64_t)fny * (2 * Z + dz));
                if (!fmask[f]) continue;
                ++k;
                sr += frho[f];
                su[0] += fu[f];
                su[1] += fu[fn + f];
                su[2] += fu[2 * fn + f];
            }
    const float inv = k ? 1.0f / (float)k : 0.0f;
    crho[c] = sr * inv;
    cu[c] = su[0] * inv;
    cu[cn + c] = su[1] * inv;
    cu[2 * cn + c] = su[2] * inv;
}

int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

namespace lbm {
// host-side helpers shared with lbm_domain.cu
lbm_status nn_fail(lbm_status s, const std::string& msg)
{
    set_last_error(msg.c_str());
    return s;
}
}  // namespace lbm

struct lbm_corrector {
    Box box{};
    int64_t n_cells = 0, n_fluid = 0, n_tiles = 0;
    float u_scale = 0.05f, rho_scale = 0.01f, du_scale = 0.005f, clip = 2.0f;
    cudaStream_t stream = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void* ctx = nullptr;
    std::vector<void*> owned;
    uint8_t* mask = nullptr;
    int4* tiles = nullptr;
    __nv_bfloat16 *x0 = nullptr, *y1 = nullptr, *y2 = nullptr, *dO = nullptr, *dy = nullptr, *dy2 = nullptr;
    float* o4 = nullptr;
    float *rho = nullptr, *u = nullptr, *du = nullptr;  // staging on the coarse box
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr, *wt = nullptr;
    double* loss = nullptr;
    unsigned long long* count = nullptr;
    int64_t adam_t = 0;

    void* dev(size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        void* p = nullptr;
        if (alloc) p = alloc(bytes, ctx);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) owned.push_back(p);
        return p;
    }
    void release_all()
    {
        for (void* p : owned) {
            if (release) release(p, ctx);
            else if (!alloc) cudaFree(p);
        }
        owned.clear();
    }
    float* wmaster(int l) { return master + (size_t)l * (NW + CH); }
    float* bmaster(int l) { return master + (size_t)l * (NW + CH) + NW; }

    cudaError_t conv(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, int relu,
                     const __nv_bfloat16* gate, void* out, bool f32)
    {
        if (n_tiles == 0) return cudaSuccess;
        if (f32) k_conv<true><<<(int)n_tiles, 128, 0, stream>>>(in, w, bias, relu, gate, out, tiles, box);
        else k_conv<false><<<(int)n_tiles, 128, 0, stream>>>(in, w, bias, relu, gate, out, tiles, box);
        return cudaGetLastError();
    }
    cudaError_t forward(const uint8_t* cmask, const float* r, const float* uu)
    {
        k_features<<<blocks(n_cells, 256), 256, 0, stream>>>(r, uu, cmask ? cmask : mask, box, 1.0f / u_scale,
                                                             1.0f / rho_scale, x0);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = conv(x0, wb, bmaster(0), 1, nullptr, y1, false);
        if (e == cudaSuccess) e = conv(y1, wb + NW, bmaster(1), 1, nullptr, y2, false);
        if (e == cudaSuccess) e = conv(y2, wb + 2 * NW, bmaster(2), 0, nullptr, o4, true);
        return e;
    }
    // loss and gradients into `grad` (FP32, parameter layout), loss into `loss`
    cudaError_t backward(const uint8_t* mk, const float* uu, const float* ut)
    {
        cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NP, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return e;
        k_count<<<blocks(n_cells, 256), 256, 0, stream>>>(mk, n_cells, count);
        k_loss<<<blocks(n_cells, 256), 256, 0, stream>>>(o4, uu, ut, mk, box, 1.0f / du_scale, count, dO, loss);
        e = cudaGetLastError();
        const int wg = (int)std::min<int64_t>(std::max<int64_t>(n_tiles, 1), 304);
        if (e == cudaSuccess && n_tiles)
            k_wgrad<<<wg, 128, 0, stream>>>(dO, y2, tiles, (int)n_tiles, box, grad + 2 * (NW + CH), grad + 2 * (NW + CH) + NW);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = conv(dO, wt + 2 * NW, nullptr, 0, y2, dy2, false);  // dz2 = W3^T dO, gated by y2 > 0
        if (e == cudaSuccess && n_tiles)
            k_wgrad<<<wg, 128, 0, stream>>>(dy2, y1, tiles, (int)n_tiles, box, grad + (NW + CH), grad + (NW + CH) + NW);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = conv(dy2, wt + NW, nullptr, 0, y1, dy, false);  // dz1 = W2^T dz2, gated by y1 > 0
        if (e == cudaSuccess && n_tiles)
            k_wgrad<<<wg, 128, 0, stream>>>(dy, x0, tiles, (int)n_tiles, box, grad, grad + NW);
        if (e == cudaSuccess) e = cudaGetLastError();
        return e;
    }
    cudaError_t prepare()
    {
        k_prepare<<<blocks(3 * NW, 256), 256, 0, stream>>>(master, wb, wt);
        return cudaGetLastError();
    }
};

extern "C" {

int64_t lbm_corrector_num_params(void) { return NP; }

lbm_status lbm_corrector_create(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz, double u_scale,
                                double rho_scale, double du_scale, const float* params, lbm_alloc_fn alloc,
                                lbm_free_fn release, void* alloc_ctx, void* cuda_stream, lbm_corrector** out)
{
    if (!out) return nn_fail(LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!mask || !params) return nn_fail(LBM_ERR_INVALID_ARG, "NULL mask or params");
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx % 4 || ny % 4 || nz % 4)
        return nn_fail(LBM_ERR_INVALID_ARG, "the corrector's box extents must be positive multiples of 4");
    if ((int64_t)(nx + 2) * (ny + 2) * (nz + 2) * CH >= ((int64_t)1 << 31))
        return nn_fail(LBM_ERR_INVALID_ARG, "box too large for the corrector");
    if (!(u_scale > 0 && rho_scale > 0 && du_scale > 0)) return nn_fail(LBM_ERR_INVALID_ARG, "scales must be > 0");
    if ((alloc == nullptr) != (release == nullptr)) return nn_fail(LBM_ERR_INVALID_ARG, "give both allocator callbacks or neither");
    lbm_corrector* K = new (std::nothrow) lbm_corrector();
    if (!K) return nn_fail(LBM_ERR_OOM, "host allocation failed");
    K->box = Box{nx, ny, nz, nx + 2, ny + 2, nz + 2};
    K->n_cells = (int64_t)nx * ny * nz;
    K->u_scale = (float)u_scale;
    K->rho_scale = (float)rho_scale;
    K->du_scale = (float)du_scale;
    K->stream = static_cast<cudaStream_t>(cuda_stream);
    K->alloc = alloc;
    K->release = release;
    K->ctx = alloc_ctx;
    // tiles holding fluid, dilated by one tile
    const int tx = nx / 4, ty = ny / 4, tz = nz / 4;
    std::vector<uint8_t> has((size_t)tx * ty * tz, 0), use((size_t)tx * ty * tz, 0);
    for (int64_t c = 0; c < K->n_cells; ++c)
        if (mask[c]) {
            ++K->n_fluid;
            const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
            has[(size_t)(x / 4) + (size_t)tx * ((size_t)(y / 4) + (size_t)ty * (size_t)(z / 4))] = 1;
        }
    std::vector<int4> tl;
    for (int z = 0; z < tz; ++z)
        for (int y = 0; y < ty; ++y)
            for (int x = 0; x < tx; ++x) {
                bool near = false;
                for (int dz = -1; dz <= 1 && !near; ++dz)
                    for (int dy = -1; dy <= 1 && !near; ++dy)
                        for (int dx = -1; dx <= 1 && !near; ++dx) {
                            const int X = x + dx, Y = y + dy, Z = z + dz;
                            if (X < 0 || Y < 0 || Z < 0 || X >= tx || Y >= ty || Z >= tz) continue;
                            near = has[(size_t)X + (size_t)tx * ((size_t)Y + (size_t)ty * (size_t)Z)] != 0;
                        }
                if (near) tl.push_back(make_int4(4 * x, 4 * y, 4 * z, 0));
            }
    K->n_tiles = (int64_t)tl.size();
    const size_t act = (size_t)K->box.px * K->box.py * K->box.pz * CH * sizeof(__nv_bfloat16);
    const size_t cells = (size_t)K->n_cells;
    bool ok = true;
    auto D = [&](size_t bytes) {
        void* p = K->dev(bytes);
        ok = ok && p;
        return p;
    };
    K->mask = static_cast<uint8_t*>(D(cells));
    K->tiles = static_cast<int4*>(D(sizeof(int4) * std::max<size_t>(tl.size(), 1)));
    K->x0 = static_cast<__nv_bfloat16*>(D(act));
    K->y1 = static_cast<__nv_bfloat16*>(D(act));
    K->y2 = static_cast<__nv_bfloat16*>(D(act));
    K->dO = static_cast<__nv_bfloat16*>(D(act));
    K->dy = static_cast<__nv_bfloat16*>(D(act));
    K->dy2 = static_cast<__nv_bfloat16*>(D(act));
    K->o4 = static_cast<float*>(D(sizeof(float) * 4 * cells));
    K->rho = static_cast<float*>(D(sizeof(float) * cells));
    K->u = static_cast<float*>(D(sizeof(float) * 3 * cells));
    K->du = static_cast<float*>(D(sizeof(float) * 3 * cells));
    K->master = static_cast<float*>(D(sizeof(float) * NP));
    K->grad = static_cast<float*>(D(sizeof(float) * NP));
    K->m = static_cast<float*>(D(sizeof(float) * NP));
    K->v = static_cast<float*>(D(sizeof(float) * NP));
    K->wb = static_cast<__nv_bfloat16*>(D(sizeof(__nv_bfloat16) * 3 * NW));
    K->wt = static_cast<__nv_bfloat16*>(D(sizeof(__nv_bfloat16) * 3 * NW));
    K->loss = static_cast<double*>(D(sizeof(double)));
    K->count = static_cast<unsigned long long*>(D(sizeof(unsigned long long)));
    if (!ok) {
        K->release_all();
        delete K;
        return nn_fail(LBM_ERR_OOM, "allocation failed: corrector buffers");
    }
    cudaError_t e = cudaMemcpyAsync(K->mask, mask, cells, cudaMemcpyHostToDevice, K->stream);
    if (e == cudaSuccess && !tl.empty())
        e = cudaMemcpyAsync(K->tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice, K->stream);
    for (__nv_bfloat16* p : {K->x0, K->y1, K->y2, K->dO, K->dy, K->dy2})
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, act, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->o4, 0, sizeof(float) * 4 * cells, K->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(K->master, params, sizeof(float) * NP, cudaMemcpyHostToDevice, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->m, 0, sizeof(float) * NP, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->v, 0, sizeof(float) * NP, K->stream);
    if (e == cudaSuccess) e = K->prepare();
    if (e == cudaSuccess) e = cudaStreamSynchronize(K->stream);
    if (e != cudaSuccess) {
        K->release_all();
        delete K;
        return nn_fail(LBM_ERR_CUDA, std::string("corrector set-up: ") + cudaGetErrorString(e));
    }
    *out = K;
    return LBM_OK;
}

lbm_status lbm_corrector_get_params(lbm_corrector* K, float* params)
{
    if (!K || !params) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(params, K->master, sizeof(float) * NP, cudaMemcpyDeviceToHost, K->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(K->stream);
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("get params: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_corrector_set_params(lbm_corrector* K, const float* params)
{
    if (!K || !params) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(K->master, params, sizeof(float) * NP, cudaMemcpyHostToDevice, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->m, 0, sizeof(float) * NP, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->v, 0, sizeof(float) * NP, K->stream);
    if (e == cudaSuccess) e = K->prepare();
    if (e == cudaSuccess) e = cudaStreamSynchronize(K->stream);
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("set params: ") + cudaGetErrorString(e));
    K->adam_t = 0;
    return LBM_OK;
}

lbm_status lbm_corrector_forward(lbm_corrector* K, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                 const float* u, float* du)
{
    if (!K || !rho || !u || !du) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = K->forward(mask, rho, u);
    const uint8_t* om = out_mask ? out_mask : (mask ? mask : K->mask);
    if (e == cudaSuccess) {
        k_output<<<blocks(K->n_cells, 256), 256, 0, K->stream>>>(K->o4, om, K->n_cells, K->du_scale, K->clip, du);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("corrector forward: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_corrector_gradients(lbm_corrector* K, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                   const float* u, const float* u_target, float* grad, double* loss)
{
    if (!K || !rho || !u || !u_target || !grad || !loss) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = K->forward(mask, rho, u);
    if (e == cudaSuccess) e = K->backward(out_mask ? out_mask : (mask ? mask : K->mask), u, u_target);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, K->grad, sizeof(float) * NP, cudaMemcpyDeviceToHost, K->stream);
    double l = 0.0;
    unsigned long long cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, K->loss, sizeof(double), cudaMemcpyDeviceToHost, K->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, K->count, sizeof(cnt), cudaMemcpyDeviceToHost, K->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(K->stream);
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("corrector gradients: ") + cudaGetErrorString(e));
    *loss = cnt ? l / (3.0 * (double)cnt) : 0.0;
    return LBM_OK;
}

lbm_status lbm_corrector_train_step(lbm_corrector* K, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                    const float* u, const float* u_target, double lr, double* loss)
{
    if (!K || !rho || !u || !u_target) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (!(lr > 0.0)) return nn_fail(LBM_ERR_INVALID_ARG, "lr must be > 0");
    cudaError_t e = K->forward(mask, rho, u);
    if (e == cudaSuccess) e = K->backward(out_mask ? out_mask : (mask ? mask : K->mask), u, u_target);
    K->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.0f - std::pow(b1, (float)K->adam_t), bc2 = 1.0f - std::pow(b2, (float)K->adam_t);
    if (e == cudaSuccess) {
        k_adam<<<blocks(NP, 256), 256, 0, K->stream>>>(K->master, K->grad, K->m, K->v, NP, (float)lr, b1, b2, 1e-8f,
                                                       bc1, bc2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = K->prepare();
    double l = 0.0;
    unsigned long long cnt = 0;
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(&l, K->loss, sizeof(double), cudaMemcpyDeviceToHost, K->stream);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(&cnt, K->count, sizeof(cnt), cudaMemcpyDeviceToHost, K->stream);
    if (e == cudaSuccess && loss) e = cudaStreamSynchronize(K->stream);
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("corrector train step: ") + cudaGetErrorString(e));
    if (loss) *loss = cnt ? l / (3.0 * (double)cnt) : 0.0;
    return LBM_OK;
}

lbm_status lbm_corrector_apply(lbm_corrector* K, lbm_domain* dom, const uint8_t* mask, const uint8_t* out_mask,
                               double gain)
{
    if (!K || !dom) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (!(gain > 0.0 && gain <= 1.0)) return nn_fail(LBM_ERR_INVALID_ARG, "gain must lie in (0, 1]");
    lbm_info I{};
    lbm_get_info(dom, &I);
    if (I.nx != K->box.nx || I.ny != K->box.ny || I.nz != K->box.nz)
        return nn_fail(LBM_ERR_INVALID_ARG, "the domain's box differs from the corrector's");
    lbm_status s = lbm_get_macroscopic(dom, K->rho, K->u, 1, 1);
    if (s) return s;
    cudaError_t e = K->forward(mask, K->rho, K->u);
    const uint8_t* om = out_mask ? out_mask : (mask ? mask : K->mask);
    if (e == cudaSuccess) {
        k_output<<<blocks(K->n_cells, 256), 256, 0, K->stream>>>(K->o4, om, K->n_cells, (float)(K->du_scale * gain),
                                                                 K->clip, K->du);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("corrector apply: ") + cudaGetErrorString(e));
    return lbm_apply_velocity_correction(dom, K->du, 1);
}

void lbm_corrector_destroy(lbm_corrector* K)
{
    if (!K) return;
    cudaStreamSynchronize(K->stream);
    K->release_all();
    delete K;
}

lbm_status lbm_restrict(const float* fine_rho, const float* fine_u, const uint8_t* fine_mask, int32_t fnx, int32_t fny,
                        int32_t fnz, float* coarse_rho, float* coarse_u, void* cuda_stream)
{
    if (!fine_rho || !fine_u || !fine_mask || !coarse_rho || !coarse_u) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (fnx <= 0 || fny <= 0 || fnz <= 0 || fnx % 2 || fny % 2 || fnz % 2)
        return nn_fail(LBM_ERR_INVALID_ARG, "fine extents must be positive and even");
    const int64_t cn = (int64_t)(fnx / 2) * (fny / 2) * (fnz / 2);
    k_restrict<<<blocks(cn, 256), 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(fine_rho, fine_u, fine_mask, fnx, fny,
                                                                                     fnz, coarse_rho, coarse_u);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("restrict: ") + cudaGetErrorString(e));
    return LBM_OK;
}

}  // extern "C"
