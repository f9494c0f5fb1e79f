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
//   * Convolution = implicit GEMM on the 5th-generation tensor cores (k_conv_tc): tcgen05.mma
//     with the accumulator in tensor memory, operands staged in shared memory by TMA, a CTA per
//     8 x 16 x 1 slab (M = 128 cells, N = 16 output channels, K = 27 offsets x 16 input
//     channels).  The data-gradient is the same kernel with the flipped, transposed kernel and
//     a ReLU gate.  The weight-gradient is a GEMM over cells (K) whose M stacks the offsets along
//     x with the input channels (k_wgrad_tc, also tcgen05): the three x-shifted copies of each
//     halo row are transposed into shared memory so that every operand is a plain canonical
//     layout, and the per-CTA partial sums are added in a fixed order.
#include <cuda.h>
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

// du = du_scale * clamp(O[0:3], -clip, clip) at the masked cells of the slabs, 0 at their other
// cells (three planes; the caller zeroes the rest of the box).  The clamp lets a NaN through
// (fminf/fmaxf would turn it into -clip): a network that has gone non-finite must make the
// corrected state non-finite, which the caller's fallback detects, not apply a full-size
// correction everywhere.
__device__ __forceinline__ float clamp_keep_nan(float o, float clip)
{
    return o > clip ? clip : (o < -clip ? -clip : o);
}

// ------------------------------------------------------------------------------ tcgen05 conv
// out[p][co] = act(sum_o sum_ci w[o][co][ci] in[p + o][ci] + bias[co]), zeroed where gate <= 0,
// as an implicit GEMM on the 5th-generation tensor cores.  A slab is 8 (x) x 16 (y) x 1 (z)
// cells: M = 128 rows (cell x + 8 y), N = 16 output channels, K = 27 offsets x 16 input
// channels, i.e. 27 tcgen05.mma (kind::f16, BF16 in, FP32 accumulator of 128 lanes x 16 columns
// in tensor memory) issued by one thread.  The CTAs (128 threads) are persistent and walk over
// slabs blockIdx.x, + gridDim.x, ...: the weights are staged once per CTA, the halo of the next
// slab is loaded into the other of two buffers, and two accumulators alternate, so the 27 MMAs
// of slab j run while the epilogue of slab j - 1 drains and the halo of slab j + 1 arrives.
//   * The slab's halo (10 x 18 x 3 cells) comes in by two TMA tile loads of the channels-last
//     padded activations (a 4-D tensor map, box 8 channels x 10 x 18 x 3), one per group of 8
//     channels, so shared memory holds two "planes" of 16 bytes per cell.  For offset o the A
//     operand is a K-major, non-swizzled canonical layout read straight out of those planes:
//     8-row core matrices are 8 consecutive cells along x (16 B apart), core matrices along M
//     are the 16 y rows (160 B apart), and the two K core matrices are the two planes.  No
//     gather, no copy: the 27 descriptors differ only in their start address.
//   * B (the 27 weight blocks, N x K = 16 x 16) is stored in global memory in the same canonical
//     layout (core matrix (n-group, k-group) at 128-byte steps; k_prepare writes it) and comes in
//     with the first halo by one bulk copy.
//   * The epilogue reads each row back with tcgen05.ld (warp w owns lanes 32w..32w+31), adds the
//     bias, applies ReLU and the gate, and writes 32 bytes per cell.
// Every wait (TMA, MMA completion) is bounded; on a timeout the CTA flags the error, waits for
// what it issued, frees its tensor memory and returns.
constexpr int SL_X = 8, SL_Y = 16;                      // slab = M = 128 cells
constexpr int HX = SL_X + 2, HY = SL_Y + 2, HZ = 3;     // halo
constexpr uint32_t PLANE_BYTES = HX * HY * HZ * 16;     // 8640: one TMA box
constexpr uint32_t PLANE_STRIDE = 8704;                 // 128-byte aligned plane step
constexpr uint32_t HALO_BYTES = 2 * PLANE_STRIDE;       // one halo buffer: two planes
constexpr uint32_t W_OFF = 2 * HALO_BYTES;              // weights after the two halo buffers
constexpr uint32_t W_BYTES = 27 * 512;                  // one layer's weights, BF16
constexpr uint32_t CONV_SMEM = W_OFF + W_BYTES;         // 48640 B
constexpr int CONV_CTAS_PER_SM = 4;
constexpr int TC_WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128, N = 16
constexpr uint32_t CONV_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t phase)
{
    for (int it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(su32(bar)), "r"(phase)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Output of a convolution: BF16 activations (padded, channels-last), FP32 O[0:4] (compact float4
// per cell), or the velocity correction du = scale clamp(O[0:3]) at the cells of `mask` (0 at the
// slabs' other cells; three planes) -- the last layer of an inference with the output step fused.
enum ConvOut { OUT_BF16 = 0, OUT_F32 = 1, OUT_DU = 2 };
struct DuArgs {
    const uint8_t* mask;
    float scale, clip;
};

template <int OUT>
__global__ void __launch_bounds__(128)
    k_conv_tc(const __grid_constant__ CUtensorMap tin, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
              int relu, const __nv_bfloat16* __restrict__ gate, void* __restrict__ out, const int4* __restrict__ slabs,
              int n_slabs, Box b, unsigned int* __restrict__ err, DuArgs dua)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_tma[2], bar_mma[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    const int J = (n_slabs - (int)blockIdx.x + G - 1) / G;  // slabs of this CTA (>= 1)
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_tma[k])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_mma[k])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // two accumulators of 16 columns, at columns 0 and 32
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    // halo of slab j into buffer j & 1: padded coordinates (x0, y0, z) .. + (9, 17, 2), channels
    // 0-7 and 8-15 (issued by thread 0)
    // (slab 0 also brings the weights: one bulk copy, already in the shared-memory layout)
    auto load_halo = [&](int j) {
        const int4 sl = slabs[blockIdx.x + j * G];
        uint64_t* bar = &bar_tma[j & 1];
        unsigned char* dst = smem + (j & 1) * HALO_BYTES;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
                     "r"(2u * PLANE_BYTES + (j == 0 ? W_BYTES : 0u))
                     : "memory");
        if (j == 0)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    su32(smem + W_OFF)),
                "l"(w), "r"(W_BYTES), "r"(su32(bar))
                : "memory");
#pragma unroll
        for (int c = 0; c < 2; ++c)
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5}], [%6];" ::"r"(su32(dst + c * PLANE_STRIDE)),
                "l"(reinterpret_cast<uint64_t>(&tin)), "r"(8 * c), "r"(sl.x), "r"(sl.y), "r"(sl.z), "r"(su32(bar))
                : "memory");
    };
    if (tid == 0) {
        load_halo(0);
        if (J > 1) load_halo(1);
    }
    const uint32_t tbase = tmem_base;
    float bz[CH];
#pragma unroll
    for (int co = 0; co < CH; ++co) bz[co] = bias ? __ldg(bias + co) : 0.0f;
    // epilogue of slab j: accumulator j & 1 -> bias, ReLU, gate -> output
    auto epilogue = [&](int j) {
        const int4 sl = slabs[blockIdx.x + j * G];
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tbase + 32u * (uint32_t)(j & 1) + ((uint32_t)(warp * 32) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int m = warp * 32 + lane;
        const int x = sl.x + (m & 7), y = sl.y + (m >> 3), z = sl.z;
        if (x < b.nx && y < b.ny) {
            float v[CH];
            const size_t pc = pidx(b, x, y, z);
            uint4 gw[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
            if (gate) {  // the gate's 16 channels of this cell, two 16-byte loads
                gw[0] = __ldg(reinterpret_cast<const uint4*>(gate + pc * CH));
                gw[1] = __ldg(reinterpret_cast<const uint4*>(gate + pc * CH) + 1);
            }
            const uint32_t* g32 = reinterpret_cast<const uint32_t*>(gw);
#pragma unroll
            for (int co = 0; co < CH; ++co) {
                float t = __uint_as_float(r[co]) + bz[co];
                if (relu) t = fmaxf(t, 0.0f);
                const uint32_t gb = (co & 1) ? (g32[co >> 1] & 0xFFFF0000u) : (g32[co >> 1] << 16);
                if (gate && !(__uint_as_float(gb) > 0.0f)) t = 0.0f;
                v[co] = t;
            }
            const size_t c = ((size_t)z * b.ny + y) * b.nx + x;
            if (OUT == OUT_F32) {
                *reinterpret_cast<float4*>(static_cast<float*>(out) + c * 4) = make_float4(v[0], v[1], v[2], v[3]);
            } else if (OUT == OUT_DU) {
                const size_t n = (size_t)b.nx * b.ny * b.nz;
                const bool on = dua.mask[c] != 0;
                float* du = static_cast<float*>(out);
#pragma unroll
                for (int k = 0; k < 3; ++k) du[k * n + c] = on ? clamp_keep_nan(v[k], dua.clip) * dua.scale : 0.0f;
            } else {
                uint32_t pk[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
                    pk[k] = *reinterpret_cast<const uint32_t*>(&h);
                }
                uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + pc * CH);
                dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };
    // give up: flag the error, wait (bounded) for the halo loads t0..t1 and the MMA groups
    // m0..m1 still in flight
    auto abandon = [&](int t0, int t1, int m0, int m1) {
        if (tid == 0) atomicOr(err, 1u);
        for (int j = t0; j <= t1 && j < J; ++j) tc_wait(&bar_tma[j & 1], (j >> 1) & 1);
        for (int j = m0 < 0 ? 0 : m0; j <= m1; ++j) tc_wait(&bar_mma[j & 1], (j >> 1) & 1);
    };
    bool ok = true;
    for (int j = 0; j < J; ++j) {
        // in flight here: halo loads j (and 1 when j = 0), MMA group j - 1
        if (!__syncthreads_and(tc_wait(&bar_tma[j & 1], (j >> 1) & 1))) {  // one decision for the CTA
            abandon(j, j == 0 ? 1 : j, j - 1, j - 1);
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // a descriptor's start field is the address / 16 (no carry out of it below 256 KB): the
            // 27 offsets' descriptors are the buffer's plus constants
            const uint64_t a0 = smem_desc(su32(smem + (j & 1) * HALO_BYTES), PLANE_STRIDE, HX * 16);
            const uint64_t w0 = smem_desc(su32(smem + W_OFF), 128, 256);
            const uint32_t d = tbase + 32u * (uint32_t)(j & 1);
#pragma unroll
            for (int o = 0; o < 27; ++o) {
                const int ox = o % 3, oy = (o / 3) % 3, oz = o / 9;
                const uint64_t ad = a0 + (uint64_t)((oz * HY + oy) * HX + ox);
                const uint64_t bd = w0 + (uint64_t)(32 * o);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, "
                    "p;\n}\n" ::"r"(d),
                    "l"(ad), "l"(bd), "r"(CONV_IDESC), "r"((uint32_t)(o > 0))
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar_mma[j & 1]))
                         : "memory");
        }
        if (j >= 1) {
            const int p = j - 1;
            // in flight here: MMA groups j - 1 and j, no halo load
            if (!__syncthreads_and(tc_wait(&bar_mma[p & 1], (p >> 1) & 1))) {
                abandon(J, J - 1, p, j);
                ok = false;
                break;
            }
            epilogue(p);
            __syncthreads();  // accumulator p & 1 read; halo buffer p & 1 consumed by MMA p
            if (tid == 0 && j + 1 < J) load_halo(j + 1);
        }
    }
    if (ok) {
        const int p = J - 1;
        if (__syncthreads_and(tc_wait(&bar_mma[p & 1], (p >> 1) & 1))) {
            epilogue(p);
        } else if (tid == 0) {
            atomicOr(err, 1u);
        }
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tbase) : "memory");
}

// Partial weight gradient of this CTA's slabs on the 5th-generation tensor cores:
// part[blockIdx.x] = (dW[o][co][ci] = sum_p dy[p][co] x[p + o][ci], db[co] = sum_p dy[p][co]) over
// the cells p of slabs blockIdx.x, + gridDim.x, ...  The sums over the CTAs are taken in a fixed
// order by k_wgrad_reduce, so that a training run is reproducible bit for bit.
//   GEMM per pair (dy, dz) of offsets along y and z: D[(s, ci)][co] = sum_k A[(s, ci)][k] B[co][k]
// with k running over the slab's cells (K = 16 per MMA: two x rows of 8 cells), A[(s, ci)][k] =
// x[cell(k) + (s - 1, dy, dz)][ci] and B[co][k] = dy[cell(k)][co]; rows s = 0, 1, 2 are the three
// offsets along x.  Both operands are K-major canonical layouts (8 x 16 B core matrices, no
// swizzle) built in shared memory: for every halo row (y, z) the 8 cells that start at x0 - 1,
// x0 and x0 + 1 are stored transposed, channel by channel ([ci][8 cells], 256 B each), one after
// the other, so the M core matrices (s, ci / 8) of one offset pair lie 128 B apart and the next
// 8 cells along K (the next x row) 768 B further.  An MMA has M = 128: rows s = 3..7 read the
// following halo rows and are discarded.  The nine accumulators (16 columns each) stay in tensor
// memory over all the CTA's slabs; two staging buffers let the threads transpose slab j + 1 while
// the 72 MMAs of slab j run.  Every wait is bounded; on a timeout the CTA flags `err`, waits for
// what it issued, frees its tensor memory and returns.
constexpr int WG_CTAS = 304;                           // weight-gradient CTAs (2 per SM): the partial buffer's depth
constexpr int WG_HROWS = HY * HZ;                      // 54 halo rows (y, z) of a slab
constexpr uint32_t WG_ROW = 3 * 256;                   // one halo row: three shifted copies
constexpr uint32_t WG_A = (WG_HROWS + 2) * WG_ROW;     // + 2 rows read only by the discarded M rows
constexpr uint32_t WG_B = SL_Y * 256;                  // dy of the slab: 16 x rows of [co][8 cells]
constexpr uint32_t WG_BUF = WG_A + WG_B;               // 47104
constexpr uint32_t WG_SMEM = 2 * WG_BUF;               // 94208
// furthest byte an MMA reads in a buffer: A of the last offset pair's last K step
static_assert((uint32_t)(((HZ - 1) * HY + (SL_Y - 2) + 2) * WG_ROW) + WG_ROW + 15 * 128 + 128 <= WG_A,
              "weight-gradient A operand reads past its buffer");
static_assert((SL_Y - 2) * 256 + 256 + 128 + 128 <= (int)WG_B, "weight-gradient B operand reads past its buffer");

__global__ void __launch_bounds__(128)
    k_wgrad_tc(const __nv_bfloat16* __restrict__ dy, const __nv_bfloat16* __restrict__ x,
               const int4* __restrict__ slabs, int n_slabs, Box b, float* __restrict__ part,
               unsigned int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_mma[2];
    __shared__ uint32_t tmem_base;
    __shared__ float sdb[128][4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    const int J = (n_slabs - (int)blockIdx.x + G - 1) / G;  // slabs of this CTA (>= 1)
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_mma[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_mma[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // nine accumulators of 16 columns at columns 0, 16, ..., 128
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    const uint32_t tbase = tmem_base;
    const uint32_t* x32 = reinterpret_cast<const uint32_t*>(x);
    const uint32_t* dy32 = reinterpret_cast<const uint32_t*>(dy);
    // lane l holds, of an 8-cell x 8-channel block, cell l / 4 and channels 2 (l % 4), + 1 (one
    // 32-bit word of the channels-last data); stmatrix .trans writes the block channel by channel
    // (16 B rows of 8 cells), the canonical core-matrix rows
    const int ci8 = lane >> 2, cpw = lane & 3;
    float db[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};  // bias gradient of channels 8 g + 2 cpw + h
    // slab j's operands into buffer j & 1: warp w transposes halo rows w, w + 4, ... and x rows
    // w, w + 4, ... of dy.  Every load of the slab is issued before the first store, so the
    // warp waits for one memory latency per slab, not one per row.
    constexpr int RW = (WG_HROWS + 3) / 4;  // halo rows per warp (14; warps 2 and 3 have 13)
    auto stage = [&](int j) {
        const int4 sl = slabs[blockIdx.x + j * G];
        const uint32_t A = su32(smem + (j & 1) * WG_BUF), B = A + WG_A;
        uint32_t v[RW][3][2], u[SL_Y / 4][2];
#pragma unroll
        for (int i = 0; i < RW; ++i) {
            const int r = warp + 4 * i;
            const int Y = sl.y + r % HY, Z = sl.z + r / HY;  // padded coordinates
            const bool row_ok = r < WG_HROWS && Y < b.py && Z < b.pz;
#pragma unroll
            for (int sx = 0; sx < 3; ++sx) {
                const int X = sl.x + ci8 + sx;
                const bool ok = row_ok && X < b.px;
                const size_t c8 = ok ? (((size_t)Z * b.py + Y) * b.px + X) * (CH / 2) : 0;
                v[i][sx][0] = ok ? __ldg(x32 + c8 + cpw) : 0u;
                v[i][sx][1] = ok ? __ldg(x32 + c8 + 4 + cpw) : 0u;
            }
        }
#pragma unroll
        for (int i = 0; i < SL_Y / 4; ++i) {
            const int X = sl.x + ci8, Y = sl.y + warp + 4 * i;
            const bool ok = X < b.nx && Y < b.ny;
            const size_t c8 = ok ? pidx(b, X, Y, sl.z) * (CH / 2) : 0;
#pragma unroll
            for (int g = 0; g < 2; ++g) u[i][g] = ok ? __ldg(dy32 + c8 + 4 * g + cpw) : 0u;
        }
#pragma unroll
        for (int i = 0; i < RW; ++i) {
            const int r = warp + 4 * i;
            if (r >= WG_HROWS) break;  // warp-uniform
            // blocks (sx, g) at row + 256 sx + 128 g: lane l gives the address of row l % 8 of
            // block l / 8 (x4: sx = 0, 1) and of block 4 + l / 8 (x2: sx = 2, lanes 0-15)
            const uint32_t row = A + (uint32_t)r * WG_ROW + 16u * (uint32_t)lane;
            asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(row),
                         "r"(v[i][0][0]), "r"(v[i][0][1]), "r"(v[i][1][0]), "r"(v[i][1][1])
                         : "memory");
            asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1, %2};" ::"r"(row + 512u * (lane < 16)),
                         "r"(v[i][2][0]), "r"(v[i][2][1])
                         : "memory");
        }
#pragma unroll
        for (int i = 0; i < SL_Y / 4; ++i) {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                db[g][0] += __uint_as_float(u[i][g] << 16);
                db[g][1] += __uint_as_float(u[i][g] & 0xFFFF0000u);
            }
            const uint32_t row = B + (uint32_t)(warp + 4 * i) * 256u + 16u * (uint32_t)(lane & 15);
            asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1, %2};" ::"r"(row), "r"(u[i][0]),
                         "r"(u[i][1])
                         : "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
    };
    // the 72 MMAs of slab j (thread 0); a descriptor's start field is the address / 16 (no carry
    // out of it below 256 KB), so the operands' descriptors are the buffer's plus constants
    auto issue = [&](int j) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t A = su32(smem + (j & 1) * WG_BUF), B = A + WG_A;
        const uint64_t a0 = smem_desc(A, WG_ROW, 128), b0 = smem_desc(B, 256, 128);
        const uint32_t acc = j > 0 ? 1u : 0u;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
#pragma unroll
            for (int k = 0; k < SL_Y / 2; ++k) {
                const uint64_t ad = a0 + (uint64_t)(((a / 3) * HY + 2 * k + a % 3) * (int)(WG_ROW >> 4));
                const uint64_t bd = b0 + (uint64_t)(k * (512 >> 4));
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, "
                    "p;\n}\n" ::"r"(tbase + 16u * (uint32_t)a),
                    "l"(ad), "l"(bd), "r"(CONV_IDESC), "r"(k > 0 ? 1u : acc)
                    : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&bar_mma[j & 1]))
                     : "memory");
    };
    bool ok = true;
    int issued = 0;  // MMA groups issued (the same count in every thread)
    for (int j = 0; j < J; ++j) {
        if (j >= 2) {  // buffer j & 1 is free once the MMAs of slab j - 2 are done
            const int p = j - 2;
            if (!__syncthreads_and(tc_wait(&bar_mma[p & 1], (p >> 1) & 1))) {
                ok = false;
                break;
            }
        }
        stage(j);
        __syncthreads();
        if (tid == 0) issue(j);
        ++issued;
    }
    // the last group's completion covers every MMA issued before it
    if (ok && !__syncthreads_and(tc_wait(&bar_mma[(J - 1) & 1], ((J - 1) >> 1) & 1))) ok = false;
    if (!ok) {
        if (tid == 0) atomicOr(err, 1u);
        // bounded waits for the groups that may still be in flight, so that the tensor memory is
        // idle when it is freed
        for (int p = issued >= 2 ? issued - 2 : 0; p < issued; ++p) tc_wait(&bar_mma[p & 1], (p >> 1) & 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float* dW = part + (size_t)blockIdx.x * (NW + CH);
        if (warp < 2) {
            const int m = warp * 32 + lane, sx = m >> 4, ci = m & 15;
#pragma unroll 1
            for (int a = 0; a < 9; ++a) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(tbase + 16u * (uint32_t)a + ((uint32_t)(warp * 32) << 16)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (sx < 3) {
                    const int o = sx + 3 * (a % 3) + 9 * (a / 3);
#pragma unroll
                    for (int co = 0; co < CH; ++co) dW[(o * CH + co) * CH + ci] = __uint_as_float(r[co]);
                }
            }
        }
        sdb[tid][0] = db[0][0];
        sdb[tid][1] = db[0][1];
        sdb[tid][2] = db[1][0];
        sdb[tid][3] = db[1][1];
        __syncthreads();
        if (tid < CH) {  // channel 8 g + 2 c + h: the threads with tid' % 4 = c, in increasing tid'
            const int g = tid >> 3, c = (tid >> 1) & 3, h = tid & 1;
            float acc = 0.0f;
            for (int t = c; t < 128; t += 4) acc += sdb[t][2 * g + h];
            dW[NW + tid] = acc;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase) : "memory");
}

// out[k] = sum over the n_part partial gradients of part[p][k] (weights and biases of one layer,
// NW + CH values), in a fixed order: a CTA takes 32 consecutive k; its thread (c, k) adds the
// partials p = c, c + 8, ... in increasing p, and the eight chunk sums are then added in
// increasing c.
constexpr int WR_K = 32, WR_C = 8;
__global__ void __launch_bounds__(WR_K * WR_C)
    k_wgrad_reduce(const float* __restrict__ part, int n_part, float* __restrict__ out)
{
    __shared__ float cs[WR_C][WR_K];
    const int kk = threadIdx.x % WR_K, c = threadIdx.x / WR_K;
    const int k = blockIdx.x * WR_K + kk;
    float s = 0.0f;
    if (k < NW + CH) {
#pragma unroll 8
        for (int p = c; p < n_part; p += WR_C) s += part[(size_t)p * (NW + CH) + k];
    }
    cs[c][kk] = s;
    __syncthreads();
    if (c == 0 && k < NW + CH) {
        float t = cs[0][kk];
#pragma unroll
        for (int q = 1; q < WR_C; ++q) t += cs[q][kk];
        out[k] = t;
    }
}

// The elementwise kernels of the corrector run over the slabs of the convolutions (one CTA of
// 128 threads per 8 x 16 x 1 slab), which cover every cell a call's masks can select (they lie
// inside the creation mask) -- a tenth of the coarse box or less; the other cells of the padded
// activations and of the output gradient stay zero from creation.
__device__ __forceinline__ bool slab_cell(const int4* slabs, const Box& b, int& x, int& y, int& z, int64_t& c)
{
    const int4 sl = slabs[blockIdx.x];
    x = sl.x + (int)(threadIdx.x & 7u);
    y = sl.y + (int)(threadIdx.x >> 3);
    z = sl.z;
    c = ((int64_t)z * b.ny + y) * b.nx + x;
    return x < b.nx && y < b.ny;
}

// Input features on the padded box: u / u_scale (3), (rho - 1) / rho_scale, fluid mask, zeros.
__global__ void __launch_bounds__(128) k_features(const float* __restrict__ rho, const float* __restrict__ u,
                                                  const uint8_t* __restrict__ mask, Box b, float inv_us, float inv_rs,
                                                  __nv_bfloat16* __restrict__ x0, const int4* __restrict__ slabs)
{
    int x, y, z;
    int64_t c;
    if (!slab_cell(slabs, b, x, y, z, c)) return;
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
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

// Loss = mean over fluid cells and components of (O - T)^2, T = (u_target - u) / du_scale;
// dO = 2 (O - T) / N at fluid cells (BF16, padded, channels 0..2).
__global__ void __launch_bounds__(128) k_count(const uint8_t* __restrict__ mask, Box b, const int4* __restrict__ slabs,
                                               unsigned long long* __restrict__ count)
{
    int x, y, z;
    int64_t c;
    const bool in = slab_cell(slabs, b, x, y, z, c);
    const unsigned int ballot = __ballot_sync(0xffffffffu, in && mask[c] != 0);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(count, (unsigned long long)__popc(ballot));
}

__global__ void __launch_bounds__(128) k_loss(const float* __restrict__ o4, const float* __restrict__ u,
                                              const float* __restrict__ ut, const uint8_t* __restrict__ mask, Box b,
                                              float inv_du, const unsigned long long* __restrict__ count,
                                              __nv_bfloat16* __restrict__ dO, double* __restrict__ loss,
                                              const int4* __restrict__ slabs)
{
    __shared__ double sh[4];
    const float two_over_n = *count ? 2.0f / (3.0f * (float)*count) : 0.0f;
    const int64_t n = (int64_t)b.nx * b.ny * b.nz;
    int x, y, z;
    int64_t c;
    double part = 0.0;
    if (slab_cell(slabs, b, x, y, z, c)) {
        // every slab cell is written (zero off the mask), so that a mask differing from the
        // previous call's leaves no stale gradient behind
        __nv_bfloat16* d = dO + pidx(b, x, y, z) * CH;
        const bool on = mask[c] != 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float r = 0.0f;
            if (on) {
                r = o4[c * 4 + k] - (ut[k * n + c] - u[k * n + c]) * inv_du;
                part += (double)r * r;
            }
            d[k] = __float2bfloat16_rn(two_over_n * r);
        }
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(loss, (sh[0] + sh[1]) + (sh[2] + sh[3]));
}

// Position of weight (o, co, ci) in a layer's BF16 block, which is the convolution's shared-memory
// layout (copied in as is): block o of 512 B holds the core matrices (co / 8, ci / 8) at 128-byte
// steps, row co % 8 at 16-byte steps, ci % 8 within the row.
__device__ __forceinline__ int w_layout(int o, int co, int ci)
{
    return o * 256 + (2 * (co >> 3) + (ci >> 3)) * 64 + (co & 7) * 8 + (ci & 7);
}

// BF16 forward weights and, for layers 2 and 3, the data-gradient kernels
// wt[o'][ci][co] = w[26 - o'][co][ci] (flipped offsets, transposed channels), both in w_layout.
__global__ void k_prepare(const float* __restrict__ master, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * NW) return;
    const int l = i / NW, r = i % NW;
    const int o = r / (CH * CH), co = (r / CH) % CH, ci = r % CH;
    const float v = master[l * (NW + CH) + r];
    wb[l * NW + w_layout(o, co, ci)] = __float2bfloat16_rn(v);
    wt[l * NW + w_layout(26 - o, ci, co)] = __float2bfloat16_rn(v);
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

// 4-D tensor map over a channels-last padded activation buffer [pz][py][px][16] (BF16) whose
// box is one slab halo of one 8-channel group: 8 channels x 10 x 18 x 3 cells.
cudaError_t encode_halo_map(CUtensorMap* tm, const void* base, const Box& b)
{
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = reinterpret_cast<Encode>(fn);
    }
    const cuuint64_t dims[4] = {(cuuint64_t)CH, (cuuint64_t)b.px, (cuuint64_t)b.py, (cuuint64_t)b.pz};
    const cuuint64_t strides[3] = {(cuuint64_t)CH * 2, (cuuint64_t)b.px * CH * 2, (cuuint64_t)b.px * b.py * CH * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)HX, (cuuint32_t)HY, (cuuint32_t)HZ};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

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
    int4* slabs = nullptr;   // 8 x 16 x 1 slabs covering the 4^3 tiles with fluid, dilated by one tile
    int64_t n_slabs = 0;
    unsigned int* err = nullptr;  // set by a conv CTA whose bounded wait gave up
    cudaEvent_t ev = nullptr;     // orders the corrector's stream and a domain's stream (apply)
    CUtensorMap tmaps[5];         // halo maps of x0, y1, y2, dO, dy2 (the convolutions' inputs)
    const void* tmap_of[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    __nv_bfloat16 *x0 = nullptr, *y1 = nullptr, *y2 = nullptr, *dO = nullptr, *dy = nullptr, *dy2 = nullptr;
    float* o4 = nullptr;
    float *rho = nullptr, *u = nullptr, *du = nullptr;  // staging on the coarse box
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float* wpart = nullptr;  // [WG_CTAS][NW + CH] partial weight gradients of one layer
    __nv_bfloat16 *wb = nullptr, *wt = nullptr;
    double* loss = nullptr;
    unsigned long long* count = nullptr;
    int64_t adam_t = 0;
    int sms = 0;  // SMs of the device the corrector was created on
    uint64_t export_serial = 0;  // the domain whose zeros rho, u hold outside its fluid cells (0: none)

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
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
        for (void* p : owned) {
            if (release) release(p, ctx);
            else if (!alloc) cudaFree(p);
        }
        owned.clear();
    }
    float* wmaster(int l) { return master + (size_t)l * (NW + CH); }
    float* bmaster(int l) { return master + (size_t)l * (NW + CH) + NW; }

    cudaError_t conv(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, int relu,
                     const __nv_bfloat16* gate, void* out, int mode, DuArgs dua = DuArgs{nullptr, 0.0f, 0.0f})
    {
        if (n_slabs == 0) return cudaSuccess;
        int t = 0;
        while (t < 5 && tmap_of[t] != in) ++t;
        if (t == 5) return cudaErrorInvalidValue;
        const int grid = (int)std::min<int64_t>(n_slabs, (int64_t)sms * CONV_CTAS_PER_SM);
        auto k = mode == OUT_F32 ? k_conv_tc<OUT_F32> : mode == OUT_DU ? k_conv_tc<OUT_DU> : k_conv_tc<OUT_BF16>;
        k<<<grid, 128, CONV_SMEM, stream>>>(tmaps[t], w, bias, relu, gate, out, slabs, (int)n_slabs, box, err, dua);
        return cudaGetLastError();
    }
    // nonzero device error word (read after the stream has been synchronised)
    bool device_error()
    {
        unsigned int h = 0;
        if (cudaMemcpy(&h, err, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return true;
        if (h) cudaMemset(err, 0, sizeof(h));
        return h != 0;
    }
    // the network on the slabs: O into o4 (du == nullptr), or, for an inference, the correction
    // du = scale clamp(O[0:3]) at the cells of out_mask straight from the last layer
    cudaError_t forward(const uint8_t* cmask, const float* r, const float* uu, float* du = nullptr,
                        const uint8_t* out_mask = nullptr, float scale = 0.0f)
    {
        if (n_slabs == 0) return cudaSuccess;
        k_features<<<(unsigned)n_slabs, 128, 0, stream>>>(r, uu, cmask ? cmask : mask, box, 1.0f / u_scale,
                                                          1.0f / rho_scale, x0, slabs);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = conv(x0, wb, bmaster(0), 1, nullptr, y1, OUT_BF16);
        if (e == cudaSuccess) e = conv(y1, wb + NW, bmaster(1), 1, nullptr, y2, OUT_BF16);
        if (e == cudaSuccess && !du) e = conv(y2, wb + 2 * NW, bmaster(2), 0, nullptr, o4, OUT_F32);
        if (e == cudaSuccess && du) e = conv(y2, wb + 2 * NW, bmaster(2), 0, nullptr, du, OUT_DU, DuArgs{out_mask, scale, clip});
        return e;
    }
    // loss and gradients into `grad` (FP32, parameter layout), loss into `loss`
    cudaError_t backward(const uint8_t* mk, const float* uu, const float* ut)
    {
        cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NP, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return e;
        if (n_slabs) {
            k_count<<<(unsigned)n_slabs, 128, 0, stream>>>(mk, box, slabs, count);
            k_loss<<<(unsigned)n_slabs, 128, 0, stream>>>(o4, uu, ut, mk, box, 1.0f / du_scale, count, dO, loss, slabs);
        }
        e = cudaGetLastError();
        const int wg = (int)std::min<int64_t>(std::max<int64_t>(n_slabs, 1), WG_CTAS);
        // weight gradient of one layer: per-CTA partials, then their sum in a fixed order
        auto wgrad = [&](const __nv_bfloat16* g, const __nv_bfloat16* xin, float* out) {
            if (!n_slabs) return cudaSuccess;
            k_wgrad_tc<<<wg, 128, WG_SMEM, stream>>>(g, xin, slabs, (int)n_slabs, box, wpart, err);
            k_wgrad_reduce<<<blocks(NW + CH, WR_K), WR_K * WR_C, 0, stream>>>(wpart, wg, out);
            return cudaGetLastError();
        };
        if (e == cudaSuccess) e = wgrad(dO, y2, grad + 2 * (NW + CH));
        if (e == cudaSuccess) e = conv(dO, wt + 2 * NW, nullptr, 0, y2, dy2, OUT_BF16);  // dz2 = W3^T dO, gated by y2 > 0
        if (e == cudaSuccess) e = wgrad(dy2, y1, grad + (NW + CH));
        if (e == cudaSuccess) e = conv(dy2, wt + NW, nullptr, 0, y1, dy, OUT_BF16);  // dz1 = W2^T dz2, gated by y1 > 0
        if (e == cudaSuccess) e = wgrad(dy, x0, grad);
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
                if (near) {
                    tl.push_back(make_int4(4 * x, 4 * y, 4 * z, 0));
                    use[(size_t)x + (size_t)tx * ((size_t)y + (size_t)ty * (size_t)z)] = 1;
                }
            }
    K->n_tiles = (int64_t)tl.size();
    // slabs of 8 x 16 x 1 cells that meet a tile of that set
    std::vector<int4> sv;
    for (int z = 0; z < nz; ++z)
        for (int y0 = 0; y0 < ny; y0 += SL_Y)
            for (int x0 = 0; x0 < nx; x0 += SL_X) {
                bool any = false;
                for (int y = y0; y < std::min(ny, y0 + SL_Y) && !any; y += 4)
                    for (int x = x0; x < std::min(nx, x0 + SL_X) && !any; x += 4)
                        any = use[(size_t)(x / 4) + (size_t)tx * ((size_t)(y / 4) + (size_t)ty * (size_t)(z / 4))] != 0;
                if (any) sv.push_back(make_int4(x0, y0, z, 0));
            }
    K->n_slabs = (int64_t)sv.size();
    const size_t act = (size_t)K->box.px * K->box.py * K->box.pz * CH * sizeof(__nv_bfloat16);
    const size_t cells = (size_t)K->n_cells;
    bool ok = true;
    auto D = [&](size_t bytes) {
        void* p = K->dev(bytes);
        ok = ok && p;
        return p;
    };
    K->mask = static_cast<uint8_t*>(D(cells));
    K->slabs = static_cast<int4*>(D(sizeof(int4) * std::max<size_t>(sv.size(), 1)));
    K->err = static_cast<unsigned int*>(D(sizeof(unsigned int)));
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
    K->wpart = static_cast<float*>(D(sizeof(float) * (size_t)WG_CTAS * (NW + CH)));
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
    if (e == cudaSuccess && !sv.empty())
        e = cudaMemcpyAsync(K->slabs, sv.data(), sizeof(int4) * sv.size(), cudaMemcpyHostToDevice, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->err, 0, sizeof(unsigned int), K->stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&K->ev, cudaEventDisableTiming);
    {  // the convolutions' grid and their shared-memory sizes, once
        int dev = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&K->sms, cudaDevAttrMultiProcessorCount, dev);
        const auto smem_attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<OUT_BF16>, smem_attr, (int)CONV_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<OUT_F32>, smem_attr, (int)CONV_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<OUT_DU>, smem_attr, (int)CONV_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_wgrad_tc, smem_attr, (int)WG_SMEM);
    }
    {
        const __nv_bfloat16* ins[5] = {K->x0, K->y1, K->y2, K->dO, K->dy2};
        for (int t = 0; t < 5 && e == cudaSuccess; ++t) {
            e = encode_halo_map(&K->tmaps[t], ins[t], K->box);
            K->tmap_of[t] = ins[t];
        }
    }
    for (__nv_bfloat16* p : {K->x0, K->y1, K->y2, K->dO, K->dy, K->dy2})
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, act, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->o4, 0, sizeof(float) * 4 * cells, K->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(K->du, 0, sizeof(float) * 3 * cells, K->stream);
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
    NvtxRange nvtx_range("lbm_corrector_forward");
    if (!K || !rho || !u || !du) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    const uint8_t* om = out_mask ? out_mask : (mask ? mask : K->mask);
    // the slabs write their cells; the rest of the caller's box is zero
    cudaError_t e = cudaMemsetAsync(du, 0, sizeof(float) * 3 * K->n_cells, K->stream);
    if (e == cudaSuccess) e = K->forward(mask, rho, u, du, om, K->du_scale);
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("corrector forward: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_corrector_gradients(lbm_corrector* K, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                   const float* u, const float* u_target, float* grad, double* loss)
{
    NvtxRange nvtx_range("lbm_corrector_gradients");
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
    if (K->device_error()) return nn_fail(LBM_ERR_TIMEOUT, "a convolution gave up waiting for its copies or MMAs");
    *loss = cnt ? l / (3.0 * (double)cnt) : 0.0;
    return LBM_OK;
}

lbm_status lbm_corrector_train_step(lbm_corrector* K, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                    const float* u, const float* u_target, double lr, double* loss)
{
    NvtxRange nvtx_range("lbm_corrector_train_step");
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
    if (loss && K->device_error())
        return nn_fail(LBM_ERR_TIMEOUT, "a convolution gave up waiting for its copies or MMAs");
    if (loss) *loss = cnt ? l / (3.0 * (double)cnt) : 0.0;
    return LBM_OK;
}

lbm_status lbm_corrector_apply(lbm_corrector* K, lbm_domain* dom, const uint8_t* mask, const uint8_t* out_mask,
                               double gain)
{
    NvtxRange nvtx_range("lbm_corrector_apply");
    if (!K || !dom) return nn_fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (!(gain > 0.0 && gain <= 1.0)) return nn_fail(LBM_ERR_INVALID_ARG, "gain must lie in (0, 1]");
    lbm_info I{};
    lbm_get_info(dom, &I);
    if (I.nx != K->box.nx || I.ny != K->box.ny || I.nz != K->box.nz)
        return nn_fail(LBM_ERR_INVALID_ARG, "the domain's box differs from the corrector's");
    DomainAccess da{};
    if (!domain_access(dom, &da)) return nn_fail(LBM_ERR_INVALID_ARG, "NULL domain");
    // rho, u are exported on the domain's stream and the correction is applied there: the
    // corrector's own stream waits for the one and the domain's stream for the other.  The cells
    // that are not fluid are cleared only when the staging last held another domain's export
    // (the box is cleared once per domain, not on every call)
    cudaError_t e = enqueue_macroscopic_dense(dom, K->rho, K->u, da.serial != K->export_serial);
    K->export_serial = e == cudaSuccess ? da.serial : 0;
    if (e == cudaSuccess && da.stream != K->stream) {
        e = cudaEventRecord(K->ev, da.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(K->stream, K->ev, 0);
    }
    const uint8_t* om = out_mask ? out_mask : (mask ? mask : K->mask);
    // cells outside the slabs keep the zero of set-up
    if (e == cudaSuccess) e = K->forward(mask, K->rho, K->u, K->du, om, (float)(K->du_scale * gain));
    if (e == cudaSuccess && da.stream != K->stream) {
        e = cudaEventRecord(K->ev, K->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(da.stream, K->ev, 0);
    }
    // the correction reuses the rho, u exported above (the domain has not stepped since)
    if (e == cudaSuccess) e = enqueue_velocity_correction(dom, K->rho, K->u, K->du);
    if (e != cudaSuccess) return nn_fail(LBM_ERR_CUDA, std::string("corrector apply: ") + cudaGetErrorString(e));
    return LBM_OK;
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
    NvtxRange nvtx_range("lbm_restrict");
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
