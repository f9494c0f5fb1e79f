// lbm_device.cuh -- device code of the fused stream-collide step and its companions, templated
// on the storage precision, the streaming scheme and the launch shape.  Included by one
// translation unit per storage precision (lbm_step_fp32.cu, lbm_step_fp16.cu, lbm_step_bf16.cu).
//
// Method (Hosseini et al.):
//   LBE f_i(x + c_i, n + 1) = f_i(x, n) + Omega_i             (Sec. 2.1.1, first equation)
//   Omega = T^-1 S T (f_eq - f), central Hermite moments       (Sec. 2.1.3)
//   T f_eq = (rho, 0, ..., 0) with the full-expansion f_eq     (Eq. Hermite_coeff_eq)
//   Bouzidi interpolated bounce-back, q = |x_f - x_s| / |c|    (Sec. 2.1.4)
//
// GB300 design:
//   * Populations are SoA, pop[i][slot], slot = brick * 64 + local cell of a 4x4x4 brick; only
//     bricks with fluid (and, for the twist, their +{0,1}^3 neighbours) are stored.  One thread
//     per slot, BRICKS bricks per CTA; a warp covers half a brick and hands the brick's
//     neighbour row out with shuffles, so streaming reads no per-cell neighbour index and the
//     kernel has no CTA barrier.
//   * Two streaming schemes, same arithmetic, bitwise-equal results:
//       A-B (pull from array A, write to array B): 26 neighbour cells per update;
//       esoteric twist (in place, one array): the thread of cell x touches only the 8 cells
//       x + {0,1}^3.  On even levels it reads f_i from slot i of cell x + p_opp(i) and writes
//       f*_i to slot opp(i) of cell x + p_i; odd levels swap the two slot roles
//       (p_i = max(c_i, 0)).  Every location is read and then written by one thread only.
//   * Every lane issues all 27 loads unconditionally; halfway bounce-back is folded into the
//     address (A-B: the cell's own opposite slot; twist: the swapped slot of the same cell).
//   * A per-slot 32-bit word carries the wall mask and the cell kind, so bulk cells take no
//     boundary branch.
//   * Arithmetic is FP32 on deviations d_i = f_i - w_i throughout (moments, transforms,
//     relaxation, closures): the O(1) rest-state weights never enter a rounding.
//   * The 27x27 transform runs as three passes of nine 1-D three-point transforms
//     (T = M(u_x) (x) M(u_y) (x) M(u_z)), forward and inverse, about 500 FP32 flops per cell;
//     with the default rates (third to sixth order = 1) the forward part reduces to the moments
//     up to second order (about 350 flops per cell in all).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "lbm_internal.h"

namespace lbm {
namespace dev {

constexpr float CS2 = 1.0f / 3.0f;

// ------------------------------------------------------------------------------ LBM_DEBUG
// Built with -DLBM_DEBUG, every access of a population array, the Bouzidi q and side lists and
// the open-boundary records is checked against the array's extent first: an access out of range
// is skipped (a load gives 0) and the check's code is kept in a device flag of this translation
// unit (the first one wins), which the host reads at its next synchronising call.  Codes:
// 1 A-B pull, 2 twist load, 3 twist store, 4 A-B store, 5 Bouzidi q / side list, 6 open-boundary
// record, 7 velocity-correction update.  Without the macro every check is the constant true.
#ifdef LBM_DEBUG
static __device__ unsigned int g_debug_fault = 0u;
__device__ __forceinline__ bool dbg_in_range(uint64_t i, uint64_t n, unsigned code)
{
    if (i < n) return true;
    atomicCAS(&g_debug_fault, 0u, code);
    return false;
}
#define LBM_IN_RANGE(i, n, code) ::lbm::dev::dbg_in_range((uint64_t)(i), (uint64_t)(n), (code))
#else
#define LBM_IN_RANGE(i, n, code) true
#endif

// ------------------------------------------------------------------------------ storage
// FP32 stores d_i; FP16 / BF16 store d_i / w_i.  `load` may use the read-only path (arrays
// not written by the kernel); `load_rw` is a plain load (the in-place array).
template <int ST>
struct Store;

template <>
struct Store<LBM_STORE_FP32> {
    using T = float;
    static constexpr bool SCALED = false;  // the stored value is d itself
    static __device__ __forceinline__ float load(const void* p, int, uint32_t off)
    {
        return __ldg(static_cast<const float*>(p) + off);
    }
    static __device__ __forceinline__ float load_h(const void* p, uint32_t off) { return load(p, 0, off); }
    // with a 256-byte L2 fetch on a miss: a warp reads 128 bytes of a brick's 256-byte plane
    // row and the other half-brick warp (or the neighbour brick's shifted read) the rest, so
    // the second request finds it in L2 (measured: -3% per step cold for the two-cell kernel,
    // neutral to slightly worse for 16-bit storage, which keeps plain loads).  The asm is not
    // volatile, so the compiler may schedule it freely: every caller's stores to a location it
    // loaded depend on the loaded value.
    static __device__ __forceinline__ float load_rw(const void* p, int, uint32_t off)
    {
        float v;
        asm("ld.global.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(static_cast<const float*>(p) + off));
        return v;
    }
    static __device__ __forceinline__ float load_rw_h(const void* p, uint32_t off) { return load_rw(p, 0, off); }
    static __device__ __forceinline__ void store(void* p, int, uint32_t off, float v)
    {
        static_cast<float*>(p)[off] = v;
    }
    static __device__ __forceinline__ void store_h(void* p, uint32_t off, float v) { static_cast<float*>(p)[off] = v; }
    // v carries the factor 2^nnz(c_i) of the deferred-halving inverse transform (exact)
    static __device__ __forceinline__ void store_x(void* p, int i, uint32_t off, float v)
    {
        static_cast<float*>(p)[off] = nnz_of(i) ? v * pow2_neg(nnz_of(i)) : v;
    }
};

template <>
struct Store<LBM_STORE_FP16> {
    using T = __half;
    static __device__ __forceinline__ float load(const void* p, int i, uint32_t off)
    {
        return w_of(i) * __half2float(__ldg(static_cast<const __half*>(p) + off));
    }
    static __device__ __forceinline__ float load_rw(const void* p, int i, uint32_t off)
    {
        return w_of(i) * __half2float(static_cast<const __half*>(p)[off]);
    }
    // the stored h = d / w as a float (the caller multiplies by w_i: scale_in)
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ float load_h(const void* p, uint32_t off)
    {
        return __half2float(__ldg(static_cast<const __half*>(p) + off));
    }
    static __device__ __forceinline__ float load_rw_h(const void* p, uint32_t off)
    {
        return __half2float(static_cast<const __half*>(p)[off]);
    }
    // v already multiplied by the direction's store factor (scale_out)
    static __device__ __forceinline__ void store_h(void* p, uint32_t off, float v)
    {
        static_cast<__half*>(p)[off] = __float2half_rn(v);
    }
    static __device__ __forceinline__ void store(void* p, int i, uint32_t off, float v)
    {
        static_cast<__half*>(p)[off] = __float2half_rn(v * inv_w_of(i));
    }
    // v carries the factor 2^nnz(c_i): one multiply by the exact constant 2^-nnz / w_i
    static __device__ __forceinline__ void store_x(void* p, int i, uint32_t off, float v)
    {
        static_cast<__half*>(p)[off] = __float2half_rn(v * (inv_w_of(i) * pow2_neg(nnz_of(i))));
    }
};

template <>
struct Store<LBM_STORE_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float load(const void* p, int i, uint32_t off)
    {
        return w_of(i) * __bfloat162float(__ldg(static_cast<const __nv_bfloat16*>(p) + off));
    }
    static __device__ __forceinline__ float load_rw(const void* p, int i, uint32_t off)
    {
        return w_of(i) * __bfloat162float(static_cast<const __nv_bfloat16*>(p)[off]);
    }
    // the stored h = d / w as a float (the caller multiplies by w_i: scale_in)
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ float load_h(const void* p, uint32_t off)
    {
        return __bfloat162float(__ldg(static_cast<const __nv_bfloat16*>(p) + off));
    }
    static __device__ __forceinline__ float load_rw_h(const void* p, uint32_t off)
    {
        return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[off]);
    }
    // v already multiplied by the direction's store factor (scale_out)
    static __device__ __forceinline__ void store_h(void* p, uint32_t off, float v)
    {
        static_cast<__nv_bfloat16*>(p)[off] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ void store(void* p, int i, uint32_t off, float v)
    {
        static_cast<__nv_bfloat16*>(p)[off] = __float2bfloat16_rn(v * inv_w_of(i));
    }
    static __device__ __forceinline__ void store_x(void* p, int i, uint32_t off, float v)
    {
        static_cast<__nv_bfloat16*>(p)[off] = __float2bfloat16_rn(v * (inv_w_of(i) * pow2_neg(nnz_of(i))));
    }
};

// The multiplies around the raw accessors, with packed FP32x2 instructions where two directions
// share the factor (the same product as the per-direction load / store above, so bit-identical).
// In: d_i = w_i h_i for the 16-bit storages; the directions j and j + 18 (c_z = -1 and +1, same
// c_x, c_y) share w.
template <int ST>
__device__ __forceinline__ void scale_in(float (&d)[Q])
{
    if constexpr (Store<ST>::SCALED) {
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const float2 v = __fmul2_rn(make_float2(d[j], d[j + 18]), make_float2(w_of(j), w_of(j)));
            d[j] = v.x;
            d[j + 18] = v.y;
            d[j + 9] = d[j + 9] * w_of(j + 9);
        }
    }
}

// Out: the factor taking a post-collision d_i to the stored value -- 1/w_i for the 16-bit
// storages, times 2^-nnz(c_i) when d carries the deferred-halving factors (X).
template <int ST, bool X>
__host__ __device__ constexpr float out_factor(int i)
{
    return (Store<ST>::SCALED ? inv_w_of(i) : 1.0f) * (X ? pow2_neg(nnz_of(i)) : 1.0f);
}

// the directions 3k and 3k + 2 (c_x = -1 and +1, same c_y, c_z) share the factor
template <int ST, bool X>
__device__ __forceinline__ void scale_out(float (&d)[Q])
{
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        constexpr float one = 1.0f;
        if (out_factor<ST, X>(3 * k) != one) {
            const float c = out_factor<ST, X>(3 * k);
            const float2 v = __fmul2_rn(make_float2(d[3 * k], d[3 * k + 2]), make_float2(c, c));
            d[3 * k] = v.x;
            d[3 * k + 2] = v.y;
        }
        if (out_factor<ST, X>(3 * k + 1) != one) d[3 * k + 1] = d[3 * k + 1] * out_factor<ST, X>(3 * k + 1);
    }
}

// two cells at once (a lane of the two-cell kernel): every direction one packed multiply
template <int ST, bool X>
__device__ __forceinline__ void scale_out2(float2 (&d)[Q])
{
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (out_factor<ST, X>(i) != 1.0f) d[i] = __fmul2_rn(d[i], make_float2(out_factor<ST, X>(i), out_factor<ST, X>(i)));
}

// ------------------------------------------------------------------------------ streaming
// A-B pull: f_i(x, n) = f*_i(x - c_i, n - 1) from `src`; a wall link reads the cell's own
// opposite slot (halfway bounce-back f_i(x, n) = f*_opp(i)(x, n - 1)).
template <int ST>
__device__ __forceinline__ void fetch_ab(const void* __restrict__ src, uint32_t n, const int32_t* nbrow,
                                         uint32_t slot, uint32_t wm, float (&d)[Q])
{
    const int l = (int)(slot & (BRICK_CELLS - 1));
    const int lx = l & (BX - 1), ly = (l >> LBX) & (BY - 1), lz = l >> (LBX + LBY);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sx = lx - cx_of(i), sy = ly - cy_of(i), sz = lz - cz_of(i);
        // sx in [-1, BX]: the arithmetic shift gives the brick offset -1, 0 or +1
        const int ob = 13 + (sx >> LBX) + 3 * (sy >> LBY) + 9 * (sz >> LBZ);
        const uint32_t nb = (uint32_t)nbrow[ob];
        const uint32_t s = nb * BRICK_CELLS + (uint32_t)brick_local(sx & (BX - 1), sy & (BY - 1), sz & (BZ - 1));
        const bool wall = (wm >> i) & 1u;
        const uint32_t off = wall ? (uint32_t)(Q - 1 - i) * n + slot : (uint32_t)i * n + s;
        d[i] = LBM_IN_RANGE(off, (uint64_t)Q * n, 1) ? Store<ST>::load_h(src, off) : 0.0f;
    }
    scale_in<ST>(d);
}

// A-B pull in the step kernel: the brick's 27-entry neighbour row is held by lanes 0..26 of the
// warp (a warp covers half of one brick) and handed out with shuffles, so no CTA barrier or
// shared staging is needed.  All 32 lanes run the shuffles; only fluid lanes load.
template <int ST>
__device__ __forceinline__ void fetch_ab_shfl(const void* __restrict__ src, uint32_t n, int32_t row_lane,
                                              uint32_t slot, uint32_t wm, bool fluid, float (&d)[Q])
{
    const int l = (int)(slot & (BRICK_CELLS - 1));
    const int lx = l & (BX - 1), ly = (l >> LBX) & (BY - 1), lz = l >> (LBX + LBY);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sx = lx - cx_of(i), sy = ly - cy_of(i), sz = lz - cz_of(i);
        const int ob = 13 + (sx >> LBX) + 3 * (sy >> LBY) + 9 * (sz >> LBZ);
        const uint32_t nb = (uint32_t)__shfl_sync(0xffffffffu, row_lane, ob);
        const uint32_t s = nb * BRICK_CELLS + (uint32_t)brick_local(sx & (BX - 1), sy & (BY - 1), sz & (BZ - 1));
        const bool wall = (wm >> i) & 1u;
        const uint32_t off = wall ? (uint32_t)(Q - 1 - i) * n + slot : (uint32_t)i * n + s;
        if (fluid) d[i] = LBM_IN_RANGE(off, (uint64_t)Q * n, 1) ? Store<ST>::load_h(src, off) : 0.0f;
    }
    if (fluid) scale_in<ST>(d);
}

// Twist corner slots in the step kernel: lanes hold the brick's nb8 row (lane & 7).
__device__ __forceinline__ void corner_slots_shfl(int32_t row_lane, uint32_t slot, uint32_t (&cs)[8])
{
    const int l = (int)(slot & (BRICK_CELLS - 1));
    const int lx = l & (BX - 1), ly = (l >> LBX) & (BY - 1), lz = l >> (LBX + LBY);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int tx = lx + (e & 1), ty = ly + ((e >> 1) & 1), tz = lz + (e >> 2);
        const int ob = (tx >> LBX) | ((ty >> LBY) << 1) | ((tz >> LBZ) << 2);
        const uint32_t nb = (uint32_t)__shfl_sync(0xffffffffu, row_lane, ob);
        cs[e] = nb * BRICK_CELLS + (uint32_t)brick_local(tx & (BX - 1), ty & (BY - 1), tz & (BZ - 1));
    }
}

// Slots of the 8 cells x + e, e in {0,1}^3 (index ex + 2 ey + 4 ez), from the brick's nb8 row.
__device__ __forceinline__ void corner_slots(const int32_t* nb8, uint32_t slot, uint32_t (&cs)[8])
{
    const int l = (int)(slot & (BRICK_CELLS - 1));
    const int lx = l & (BX - 1), ly = (l >> LBX) & (BY - 1), lz = l >> (LBX + LBY);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int tx = lx + (e & 1), ty = ly + ((e >> 1) & 1), tz = lz + (e >> 2);
        const int ob = (tx >> LBX) | ((ty >> LBY) << 1) | ((tz >> LBZ) << 2);
        cs[e] = (uint32_t)nb8[ob] * BRICK_CELLS + (uint32_t)brick_local(tx & (BX - 1), ty & (BY - 1), tz & (BZ - 1));
    }
}

// Esoteric twist read at level parity P: f_i from slot (P ? opp(i) : i) of cell x + p_opp(i);
// on a wall link the other slot of the same cell, which holds f*_opp(i)(x, n - 1).
// PC >= 0 fixes the parity at compile time; with `clean` (warp-uniform: no lane of the warp has a
// wall link) every plane index is then a constant.
template <int ST, bool RW, int PC = -1>
__device__ __forceinline__ void fetch_et(const void* pop, uint32_t n, const uint32_t (&cs)[8], uint32_t wm,
                                         int parity, float (&d)[Q], bool clean = false)
{
    if (PC >= 0 && clean) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t off = (PC ? (uint32_t)(Q - 1 - i) : (uint32_t)i) * n + cs[corner_neg(i)];
            d[i] = LBM_IN_RANGE(off, (uint64_t)Q * n, 2) ? (RW ? Store<ST>::load_rw_h(pop, off) : Store<ST>::load_h(pop, off))
                                                        : 0.0f;
        }
        scale_in<ST>(d);
        return;
    }
    if (PC >= 0) parity = PC;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint32_t flip = ((uint32_t)parity ^ (wm >> i)) & 1u;
        const uint32_t dir = flip ? (uint32_t)(Q - 1 - i) : (uint32_t)i;
        const uint32_t off = dir * n + cs[corner_neg(i)];
        d[i] = LBM_IN_RANGE(off, (uint64_t)Q * n, 2) ? (RW ? Store<ST>::load_rw_h(pop, off) : Store<ST>::load_h(pop, off))
                                                    : 0.0f;
    }
    scale_in<ST>(d);
}

// Esoteric twist write after a step of parity P: f*_i to slot (P ? i : opp(i)) of cell x + p_i
// (PC >= 0: the parity fixed at compile time; X: d carries the factors 2^nnz(c_i); H: d has been
// through scale_out, the stored values as floats).
template <int ST, int PC = -1, bool X = false, bool H = false>
__device__ __forceinline__ void store_et(void* pop, uint32_t n, const uint32_t (&cs)[8], int parity,
                                         const float (&d)[Q])
{
    if (PC >= 0) {
        parity = PC;
        // with constant planes a write address equals the read address of the opposite
        // direction; an opaque copy of n keeps the compiler from holding 27 addresses live
        // through the collision (it recomputes them instead)
        asm("mov.b32 %0, %0;" : "+r"(n));
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint32_t dir = parity ? (uint32_t)i : (uint32_t)(Q - 1 - i);
        const uint32_t off = dir * n + cs[corner_pos(i)];
        if (!LBM_IN_RANGE(off, (uint64_t)Q * n, 3)) continue;
        if (H) Store<ST>::store_h(pop, off, d[i]);
        else if (X) Store<ST>::store_x(pop, i, off, d[i]);
        else Store<ST>::store(pop, i, off, d[i]);
    }
}

// ------------------------------------------------------------------------------ boundaries
// Open-boundary closure of an inlet (velocity) or outlet (density) cell on an axis-aligned face
// with inward normal n = sign e_axis, in deviation form.  Known: c.n <= 0.  With
// D = sum_{c.n=0} d + 2 sum_{c.n<0} d (and sum_{c.n=0} w + 2 sum_{c.n<0} w = 1):
//   inlet:  u.n = U phi, rho = (1 + D)/(1 - u.n);   outlet: rho = rho_out, u.n = 1 - (1 + D)/rho.
// Both are evaluated as deviations from 1 (rho - 1 = (D + u.n)/(1 - u.n),
// u.n = (rho_out - 1 - D)/rho_out), so that D is never rounded against 1.
// The nine unknowns (c.n = +1) by non-equilibrium bounce-back with the full equilibrium; since
// u has no tangential part, f_eq_i - f_eq_opp(i) = 6 w_i rho u.n.  Then the tangential momentum
// is zeroed by d_i += c_it D_t / 6, D_t = -sum_j c_jt d_j, which leaves mass and normal
// momentum unchanged.
__device__ __forceinline__ void close_open(float (&d)[Q], int kind, int axis, int sgn, float phi, float U,
                                           float rho_out, float drho_out)
{
    float D = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cn = sgn * (axis == 0 ? cx_of(i) : axis == 1 ? cy_of(i) : cz_of(i));
        if (cn == 0) D += d[i];
        if (cn < 0) D += 2.0f * d[i];
    }
    float rho, un;
    if (kind == KIND_INLET) {
        un = U * phi;
        rho = 1.0f + (D + un) / (1.0f - un);
    } else {
        rho = rho_out;
        un = (drho_out - D) / rho_out;
    }
    const float ru6 = 6.0f * rho * un;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cn = sgn * (axis == 0 ? cx_of(i) : axis == 1 ? cy_of(i) : cz_of(i));
        if (cn == 1) d[i] = d[Q - 1 - i] + w_of(i) * ru6;
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        if (t == axis) continue;
        float mom = 0.0f;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int ct = t == 0 ? cx_of(j) : t == 1 ? cy_of(j) : cz_of(j);
            if (ct == 1) mom += d[j];
            if (ct == -1) mom -= d[j];
        }
        const float corr = -mom * (1.0f / 6.0f);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cn = sgn * (axis == 0 ? cx_of(i) : axis == 1 ? cy_of(i) : cz_of(i));
            const int ct = t == 0 ? cx_of(i) : t == 1 ? cy_of(i) : cz_of(i);
            if (cn == 1 && ct != 0) d[i] += ct == 1 ? corr : -corr;
        }
    }
}

// Wall rules on top of the bounce-back already in d (Sec. 2.1.4 in pull form, beta = opp(alpha)
// pointing into the wall):
//   q <  1/2: f_a(x) = 2q f*_b(x) + (1 - 2q) f*_b(x + c_a)  [= the value pulled for b]
//   q >= 1/2: f_a(x) = f*_b(x)/(2q) + (2q - 1)/(2q) f*_a(x)
// with halfway bounce-back kept if x + c_a is not fluid in the first branch; then the open
// boundaries.  f*_a(x, n - 1) comes from the cell's own slot (A-B) or from the side buffer
// (twist: that slot is the one x + c_a pulls and overwrites in this step).  Returns the mask of
// the q >= 1/2 links, whose f*_a the twist must keep in the side buffer.
// Position of wall link i of a Bouzidi cell in the packed link lists (q, and the twist side
// buffer): the cell's entries start at its aux record and follow the set bits of its wall mask
// in direction order.
__device__ __forceinline__ uint32_t link_index(uint32_t off, uint32_t wm, int i)
{
    return off + (uint32_t)__popc(wm & ((1u << i) - 1u));
}

// aux: the cell's record (v.aux[slot]) when the caller has loaded it already, else -1
template <int ST, int SCHEME>
__device__ __forceinline__ uint32_t wall_rules(const DomainView& v, const void* src_ab, uint32_t slot,
                                               uint32_t word, const LevelArgs& a, float (&d)[Q], int32_t aux = -1)
{
    const uint32_t wm = word & WORD_WALL_MASK;
    const int kind = (int)((word >> WORD_KIND_SHIFT) & 3u);
    uint32_t half = 0u;
    if (kind == KIND_BOUZIDI) {
        const uint32_t off = (uint32_t)(aux >= 0 ? aux : v.aux[slot]);
        // A direction's rule reads d_i and, only when opp(i) has no link, d_opp(i), which no other
        // direction's rule changes: the order of the directions does not matter.  The twist takes
        // the links of nine directions at a time (their q and f*_a requested before the first is
        // used: one memory latency per group, not per link; -26% per step on a 128^3 aneurysm);
        // A-B, whose f*_a come from the other array, keeps one direction at a time (the grouped
        // form spills in its 64- to 80-register configurations and was 2% slower on the pipe).
        constexpr int GS = SCHEME == LBM_SCHEME_ESOTERIC ? 9 : 1;
#pragma unroll
        for (int g = 0; g < Q / GS; ++g) {
            float qg[GS], fg[GS];
#pragma unroll
            for (int j = 0; j < GS; ++j) {
                const int i = GS * g + j;
                const uint32_t li = link_index(off, wm, i);
                const bool has = ((wm >> i) & 1u) && LBM_IN_RANGE(li, v.n_bq, 5);
                qg[j] = has ? __ldg(v.bq + li) : 0.0f;
                // loaded whatever q is, so that the two loads do not wait on each other
                fg[j] = !has ? 0.0f
                             : (SCHEME == LBM_SCHEME_ESOTERIC)
                                   ? Store<ST>::load_rw(v.side, i, li)
                                   : Store<ST>::load(src_ab, i, (uint32_t)i * (uint32_t)v.n_slots + slot);
            }
#pragma unroll
            for (int j = 0; j < GS; ++j) {
                const int i = GS * g + j;
                const float q = qg[j], fa = fg[j];
                if (q > 0.0f) {  // 0: no link (or halfway bounce-back on this link)
                    if (q < 0.5f) {
                        if (!(wm & (1u << (Q - 1 - i)))) d[i] = 2.0f * q * d[i] + (1.0f - 2.0f * q) * d[Q - 1 - i];
                    } else {
                        const float inv2q = 0.5f / q;
                        d[i] = inv2q * d[i] + (1.0f - inv2q) * fa;
                        half |= 1u << i;
                    }
                }
            }
        }
    } else if (kind >= KIND_INLET) {
        const int64_t rec = aux >= 0 ? aux : v.aux[slot];
        if (LBM_IN_RANGE(rec, v.n_io, 6))
            close_open(d, kind, v.io_axis[rec], v.io_sign[rec], v.io_phi[rec], a.U, a.rho_out, a.drho_out);
    }
    return half;
}

// ------------------------------------------------------------------------------ collide
__device__ __forceinline__ void fwd3(float& gm, float& g0, float& gp, float u, float u2mcs)
{
    // (g(-1), g(0), g(+1)) -> central Hermite moments (m0, m1, m2) about u
    const float m0 = gm + g0 + gp;
    const float s1 = gp - gm;
    const float s2 = gp + gm;
    gm = m0;
    g0 = fmaf(-u, m0, s1);
    gp = fmaf(u2mcs, m0, fmaf(-2.0f * u, s1, s2));
}

__device__ __forceinline__ void inv3(float& m0, float& m1, float& m2, float u, float u2pcs)
{
    // (m0, m1, m2) -> (g(-1), g(0), g(+1)): raw sums S1 = g+ - g-, S2 = g+ + g-
    const float S1 = fmaf(u, m0, m1);
    const float S2 = fmaf(u2pcs, m0, fmaf(2.0f * u, m1, m2));
    const float g0 = m0 - S2;
    m0 = 0.5f * (S2 - S1);
    m2 = 0.5f * (S2 + S1);
    m1 = g0;
}

__host__ __device__ constexpr int order_of(int m) { return m % 3 + (m / 3) % 3 + m / 9; }

struct Moments {
    float rho, ux, uy, uz;
};

__device__ __forceinline__ Moments moments(const float (&d)[Q], const float g[3])
{
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (cx_of(i) == 1) jx += d[i];
        if (cx_of(i) == -1) jx -= d[i];
        if (cy_of(i) == 1) jy += d[i];
        if (cy_of(i) == -1) jy -= d[i];
        if (cz_of(i) == 1) jz += d[i];
        if (cz_of(i) == -1) jz -= d[i];
    }
    Moments m;
    m.rho = 1.0f + drho;
    const float ir = 1.0f / m.rho;
    m.ux = fmaf(jx, ir, 0.5f * g[0]);
    m.uy = fmaf(jy, ir, 0.5f * g[1]);
    m.uz = fmaf(jz, ir, 0.5f * g[2]);
    return m;
}

// CHM-MRT collision in deviation form.  With a = T(u) f, a_w = T(u) w (per axis (1, -u, u^2))
// and the post-collision moments a* (a*_0 = rho, first order rho g / 2 from the half-force
// forcing, a*_m = (1 - s_m) a_m for order >= 2 since a_eq = 0 there), the outgoing deviation
// is d* = T^-1(u) (a* - a_w), with a - a_w = T(u) d.
__device__ __forceinline__ void collide(float (&d)[Q], const LevelArgs& a)
{
    const Moments M = moments(d, a.g);
    const float ux = M.ux, uy = M.uy, uz = M.uz;
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    // forward T(u) d: passes along x, y, z
#pragma unroll
    for (int k = 0; k < 9; ++k) fwd3(d[3 * k], d[3 * k + 1], d[3 * k + 2], ux, ux2 - CS2);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int p = 0; p < 3; ++p) fwd3(d[p + 9 * r], d[p + 3 + 9 * r], d[p + 6 + 9 * r], uy, uy2 - CS2);
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int p = 0; p < 3; ++p) fwd3(d[p + 3 * q], d[p + 3 * q + 9], d[p + 3 * q + 18], uz, uz2 - CS2);
    // relaxation: b = a* - a_w
    const float ex[3] = {1.0f, -ux, ux2}, ey[3] = {1.0f, -uy, uy2}, ez[3] = {1.0f, -uz, uz2};
    const float s[7] = {0.0f, 0.0f, a.s2, a.s3, a.s4, a.s5, a.s6};
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        const int o = order_of(m);
        if (o == 1) {
            const float gk = (m == 1) ? a.g[0] : (m == 3) ? a.g[1] : a.g[2];
            const float uk = (m == 1) ? ux : (m == 3) ? uy : uz;
            d[m] = fmaf(0.5f * M.rho, gk, uk);
        } else if (o >= 2) {
            const float aw = ex[m % 3] * ey[(m / 3) % 3] * ez[m / 9];
            d[m] = (1.0f - s[o]) * d[m] - s[o] * aw;
        }
    }
    // inverse T(u)^-1
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int p = 0; p < 3; ++p) inv3(d[p + 3 * q], d[p + 3 * q + 9], d[p + 3 * q + 18], uz, uz2 + CS2);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int p = 0; p < 3; ++p) inv3(d[p + 9 * r], d[p + 3 + 9 * r], d[p + 6 + 9 * r], uy, uy2 + CS2);
#pragma unroll
    for (int k = 0; k < 9; ++k) inv3(d[3 * k], d[3 * k + 1], d[3 * k + 2], ux, ux2 + CS2);
}

// The same collision when every third- to sixth-order rate is 1 (the default): the
// post-collision moments of order >= 3 are then their equilibrium values (zero), so the forward
// transform is needed only up to second order.  rho - 1, j and the six raw second moments of d
// come from one pass of 1-D sums (S0 = g- + g0 + g+, S1 = g+ - g-, S2 = g+ + g- along x, then
// the same along y and z); the central second moments follow from them,
//   a_200 = P_xx - 2 u_x j_x + (u_x^2 - c_s^2)(rho - 1),
//   a_110 = P_xy - u_x j_y - u_y j_x + u_x u_y (rho - 1),
// and the inverse transform is unchanged.  Same arithmetic as `collide` up to rounding order.
// Lane arithmetic of the fast collision: one cell (float) or two cells at once (float2, packed
// FP32x2 instructions of sm_100+).  Every operation is an explicit round-to-nearest add,
// multiply or fused multiply-add, and the two forms apply them in the same order, so a cell
// gives bit-identical results whichever form updates it.
struct Lane1 {
    using V = float;
    static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ V neg(V a) { return -a; }
    static __device__ __forceinline__ V splat(float s) { return s; }
    static __device__ __forceinline__ V rcp1p(V drho) { return 1.0f / (1.0f + drho); }
    static __device__ __forceinline__ V one_plus(V x) { return __fadd_rn(1.0f, x); }
};
struct Lane2 {
    using V = float2;
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V neg(V a) { return make_float2(-a.x, -a.y); }
    static __device__ __forceinline__ V splat(float s) { return make_float2(s, s); }
    static __device__ __forceinline__ V rcp1p(V drho)
    {
        return make_float2(1.0f / (1.0f + drho.x), 1.0f / (1.0f + drho.y));
    }
    static __device__ __forceinline__ V one_plus(V x) { return __fadd2_rn(make_float2(1.0f, 1.0f), x); }
};

// 1-D inverse: (m0, m1, m2) -> (g(-1), g(0), g(+1)).  DEFER leaves out the halving of
// g(+-1): the outputs at +-1 come out doubled, exactly (a power of two), and since the three
// inputs of every later 1-D inverse share one such factor, each post-collision d_i leaves the
// three passes multiplied by 2^nnz(c_i), which the store removes (Store::store_x) -- for 16-bit
// storage inside the multiply by 1/w_i that it does anyway.  Bit-identical results, two fewer
// instructions per 1-D inverse.
template <class L, bool DEFER = false>
__device__ __forceinline__ void inv3_t(typename L::V& m0, typename L::V& m1, typename L::V& m2, typename L::V u,
                                       typename L::V u2pcs, typename L::V two_u)
{
    using V = typename L::V;
    const V S1 = L::fma(u, m0, m1);
    const V S2 = L::fma(u2pcs, m0, L::fma(two_u, m1, m2));
    const V g0 = L::sub(m0, S2);
    if (DEFER) {
        m0 = L::sub(S2, S1);
        m2 = L::add(S2, S1);
    } else {
        m0 = L::mul(L::splat(0.5f), L::sub(S2, S1));
        m2 = L::mul(L::splat(0.5f), L::add(S2, S1));
    }
    m1 = g0;
}

template <class L, bool DEFER = false>
__device__ __forceinline__ void collide_fast_t(typename L::V (&d)[Q], typename L::V s2, const float g[3])
{
    using V = typename L::V;
    V S0[9], S1[9], S2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        S2[k] = L::add(d[3 * k], d[3 * k + 2]);
        S0[k] = L::add(S2[k], d[3 * k + 1]);
        S1[k] = L::sub(d[3 * k + 2], d[3 * k]);
    }
    V T0[3], T1[3], T2[3], U0[3], U1[3], W[3];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
        T2[z] = L::add(S0[3 * z], S0[3 * z + 2]);
        T0[z] = L::add(T2[z], S0[3 * z + 1]);
        T1[z] = L::sub(S0[3 * z + 2], S0[3 * z]);
        U0[z] = L::add(L::add(S1[3 * z], S1[3 * z + 1]), S1[3 * z + 2]);
        U1[z] = L::sub(S1[3 * z + 2], S1[3 * z]);
        W[z] = L::add(L::add(S2[3 * z], S2[3 * z + 1]), S2[3 * z + 2]);
    }
    const V drho = L::add(L::add(T0[0], T0[1]), T0[2]);
    const V jz = L::sub(T0[2], T0[0]);
    const V Pzz = L::add(T0[2], T0[0]);
    const V jy = L::add(L::add(T1[0], T1[1]), T1[2]);
    const V Pyz = L::sub(T1[2], T1[0]);
    const V Pyy = L::add(L::add(T2[0], T2[1]), T2[2]);
    const V jx = L::add(L::add(U0[0], U0[1]), U0[2]);
    const V Pxz = L::sub(U0[2], U0[0]);
    const V Pxy = L::add(L::add(U1[0], U1[1]), U1[2]);
    const V Pxx = L::add(L::add(W[0], W[1]), W[2]);
    const V rho = L::one_plus(drho);
    const V ir = L::rcp1p(drho);
    const V ux = L::fma(jx, ir, L::splat(0.5f * g[0]));
    const V uy = L::fma(jy, ir, L::splat(0.5f * g[1]));
    const V uz = L::fma(jz, ir, L::splat(0.5f * g[2]));
    const V ux2 = L::mul(ux, ux), uy2 = L::mul(uy, uy), uz2 = L::mul(uz, uz);
    const V uxy = L::mul(ux, uy), uxz = L::mul(ux, uz), uyz = L::mul(uy, uz);
    const V k2 = L::sub(L::splat(1.0f), s2), ns2 = L::neg(s2);
    const V mcs = L::splat(-CS2);
    // central second moments of d (deviation form)
    const V a200 = L::fma(L::add(ux2, mcs), drho, L::fma(L::mul(L::splat(-2.0f), ux), jx, Pxx));
    const V a020 = L::fma(L::add(uy2, mcs), drho, L::fma(L::mul(L::splat(-2.0f), uy), jy, Pyy));
    const V a002 = L::fma(L::add(uz2, mcs), drho, L::fma(L::mul(L::splat(-2.0f), uz), jz, Pzz));
    const V a110 = L::fma(uxy, drho, L::fma(L::neg(ux), jy, L::fma(L::neg(uy), jx, Pxy)));
    const V a101 = L::fma(uxz, drho, L::fma(L::neg(ux), jz, L::fma(L::neg(uz), jx, Pxz)));
    const V a011 = L::fma(uyz, drho, L::fma(L::neg(uy), jz, L::fma(L::neg(uz), jy, Pyz)));
    // post-collision central moments of d: third and higher orders -w's moments (products of
    // the 1-D moments (1, -u, u^2) of the D1Q3 weights), second order relaxed
    const V ex[3] = {L::splat(1.0f), L::neg(ux), ux2}, ey[3] = {L::splat(1.0f), L::neg(uy), uy2},
            ez[3] = {L::splat(1.0f), L::neg(uz), uz2};
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        const int p = m % 3, q = (m / 3) % 3, r = m / 9;
        if (p + q + r < 3) continue;
        // a product with unit factors skipped (multiplication by 1 is exact)
        V aw = ex[p];
        if (q) aw = p ? L::mul(aw, ey[q]) : ey[q];
        if (r) aw = (p || q) ? L::mul(aw, ez[r]) : ez[r];
        d[m] = L::neg(aw);
    }
    d[0] = drho;
    d[1] = L::fma(L::mul(L::splat(0.5f), rho), L::splat(g[0]), ux);
    d[3] = L::fma(L::mul(L::splat(0.5f), rho), L::splat(g[1]), uy);
    d[9] = L::fma(L::mul(L::splat(0.5f), rho), L::splat(g[2]), uz);
    d[2] = L::fma(k2, a200, L::mul(ns2, ux2));
    d[6] = L::fma(k2, a020, L::mul(ns2, uy2));
    d[18] = L::fma(k2, a002, L::mul(ns2, uz2));
    d[4] = L::fma(k2, a110, L::mul(ns2, uxy));
    d[10] = L::fma(k2, a101, L::mul(ns2, uxz));
    d[12] = L::fma(k2, a011, L::mul(ns2, uyz));
    // inverse T(u)^-1: z, then y, then x
    const V zc = L::add(uz2, L::splat(CS2)), yc = L::add(uy2, L::splat(CS2)), xc = L::add(ux2, L::splat(CS2));
    const V z2 = L::mul(L::splat(2.0f), uz), y2 = L::mul(L::splat(2.0f), uy), x2 = L::mul(L::splat(2.0f), ux);
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int p = 0; p < 3; ++p) inv3_t<L, DEFER>(d[p + 3 * q], d[p + 3 * q + 9], d[p + 3 * q + 18], uz, zc, z2);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int p = 0; p < 3; ++p) inv3_t<L, DEFER>(d[p + 9 * r], d[p + 3 + 9 * r], d[p + 6 + 9 * r], uy, yc, y2);
#pragma unroll
    for (int k = 0; k < 9; ++k) inv3_t<L, DEFER>(d[3 * k], d[3 * k + 1], d[3 * k + 2], ux, xc, x2);
}

// The fast collision of one cell with packed FP32x2 instructions inside the cell: the 1-D
// sums along x and then y run on the z = -1 and z = +1 rows as pairs (their z = 0 rows alone),
// and the inverse passes along z and then y on the x = -1 and x = +1 columns as pairs (x = 0
// alone); the final pass along x mixes the members of a pair and stays scalar.  Every element
// sees the operations of collide_fast_t<Lane1> in the same order, so results are bit-identical.
template <bool DEFER = false>
__device__ __forceinline__ void collide_fast_p(float (&d)[Q], float s2, const float g[3])
{
    using L = Lane1;
    using P = Lane2;
    // x sums of row k = q + 3 r; index q, .x the row at r = 0 (k = q), .y the row at r = 2 (k = q + 6)
    float2 S0p[3], S1p[3], S2p[3];
    float S0m[3], S1m[3], S2m[3];  // rows at r = 1 (k = q + 3)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int k0 = q, k2 = q + 6, k1 = q + 3;
        const float2 gm = make_float2(d[3 * k0], d[3 * k2]), g0 = make_float2(d[3 * k0 + 1], d[3 * k2 + 1]),
                     gp = make_float2(d[3 * k0 + 2], d[3 * k2 + 2]);
        S2p[q] = P::add(gm, gp);
        S0p[q] = P::add(S2p[q], g0);
        S1p[q] = P::sub(gp, gm);
        S2m[q] = L::add(d[3 * k1], d[3 * k1 + 2]);
        S0m[q] = L::add(S2m[q], d[3 * k1 + 1]);
        S1m[q] = L::sub(d[3 * k1 + 2], d[3 * k1]);
    }
    // y sums at z = -1 and z = +1 (pairs) and z = 0
    const float2 T2p = P::add(S0p[0], S0p[2]);
    const float2 T0p = P::add(T2p, S0p[1]);
    const float2 T1p = P::sub(S0p[2], S0p[0]);
    const float2 U0p = P::add(P::add(S1p[0], S1p[1]), S1p[2]);
    const float2 U1p = P::sub(S1p[2], S1p[0]);
    const float2 Wp = P::add(P::add(S2p[0], S2p[1]), S2p[2]);
    const float T2m = L::add(S0m[0], S0m[2]);
    const float T0m = L::add(T2m, S0m[1]);
    const float T1m = L::sub(S0m[2], S0m[0]);
    const float U0m = L::add(L::add(S1m[0], S1m[1]), S1m[2]);
    const float U1m = L::sub(S1m[2], S1m[0]);
    const float Wm = L::add(L::add(S2m[0], S2m[1]), S2m[2]);
    const float T0[3] = {T0p.x, T0m, T0p.y}, T1[3] = {T1p.x, T1m, T1p.y}, T2[3] = {T2p.x, T2m, T2p.y};
    const float U0[3] = {U0p.x, U0m, U0p.y}, U1[3] = {U1p.x, U1m, U1p.y}, W[3] = {Wp.x, Wm, Wp.y};
    const float drho = L::add(L::add(T0[0], T0[1]), T0[2]);
    const float jz = L::sub(T0[2], T0[0]);
    const float Pzz = L::add(T0[2], T0[0]);
    const float jy = L::add(L::add(T1[0], T1[1]), T1[2]);
    const float Pyz = L::sub(T1[2], T1[0]);
    const float Pyy = L::add(L::add(T2[0], T2[1]), T2[2]);
    const float jx = L::add(L::add(U0[0], U0[1]), U0[2]);
    const float Pxz = L::sub(U0[2], U0[0]);
    const float Pxy = L::add(L::add(U1[0], U1[1]), U1[2]);
    const float Pxx = L::add(L::add(W[0], W[1]), W[2]);
    const float rho = L::one_plus(drho);
    const float ir = L::rcp1p(drho);
    const float ux = L::fma(jx, ir, 0.5f * g[0]);
    const float uy = L::fma(jy, ir, 0.5f * g[1]);
    const float uz = L::fma(jz, ir, 0.5f * g[2]);
    const float ux2 = L::mul(ux, ux), uy2 = L::mul(uy, uy), uz2 = L::mul(uz, uz);
    const float uxy = L::mul(ux, uy), uxz = L::mul(ux, uz), uyz = L::mul(uy, uz);
    const float k2 = L::sub(1.0f, s2), ns2 = L::neg(s2);
    const float mcs = -CS2;
    const float a200 = L::fma(L::add(ux2, mcs), drho, L::fma(L::mul(-2.0f, ux), jx, Pxx));
    const float a020 = L::fma(L::add(uy2, mcs), drho, L::fma(L::mul(-2.0f, uy), jy, Pyy));
    const float a002 = L::fma(L::add(uz2, mcs), drho, L::fma(L::mul(-2.0f, uz), jz, Pzz));
    const float a110 = L::fma(uxy, drho, L::fma(L::neg(ux), jy, L::fma(L::neg(uy), jx, Pxy)));
    const float a101 = L::fma(uxz, drho, L::fma(L::neg(ux), jz, L::fma(L::neg(uz), jx, Pxz)));
    const float a011 = L::fma(uyz, drho, L::fma(L::neg(uy), jz, L::fma(L::neg(uz), jy, Pyz)));
    const float ex[3] = {1.0f, L::neg(ux), ux2}, ey[3] = {1.0f, L::neg(uy), uy2}, ez[3] = {1.0f, L::neg(uz), uz2};
#pragma unroll
    for (int m = 0; m < Q; ++m) {
        const int p = m % 3, q = (m / 3) % 3, r = m / 9;
        if (p + q + r < 3) continue;
        float aw = ex[p];
        if (q) aw = p ? L::mul(aw, ey[q]) : ey[q];
        if (r) aw = (p || q) ? L::mul(aw, ez[r]) : ez[r];
        d[m] = L::neg(aw);
    }
    d[0] = drho;
    d[1] = L::fma(L::mul(0.5f, rho), g[0], ux);
    d[3] = L::fma(L::mul(0.5f, rho), g[1], uy);
    d[9] = L::fma(L::mul(0.5f, rho), g[2], uz);
    d[2] = L::fma(k2, a200, L::mul(ns2, ux2));
    d[6] = L::fma(k2, a020, L::mul(ns2, uy2));
    d[18] = L::fma(k2, a002, L::mul(ns2, uz2));
    d[4] = L::fma(k2, a110, L::mul(ns2, uxy));
    d[10] = L::fma(k2, a101, L::mul(ns2, uxz));
    d[12] = L::fma(k2, a011, L::mul(ns2, uyz));
    const float zc = L::add(uz2, CS2), yc = L::add(uy2, CS2), xc = L::add(ux2, CS2);
    const float z2 = L::mul(2.0f, uz), y2 = L::mul(2.0f, uy), x2 = L::mul(2.0f, ux);
    // inverse along z: columns (p, q) with p = 0 and p = 2 as pairs
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float2 m0 = make_float2(d[3 * q], d[3 * q + 2]), m1 = make_float2(d[3 * q + 9], d[3 * q + 11]),
               m2 = make_float2(d[3 * q + 18], d[3 * q + 20]);
        inv3_t<P, DEFER>(m0, m1, m2, P::splat(uz), P::splat(zc), P::splat(z2));
        d[3 * q] = m0.x, d[3 * q + 2] = m0.y, d[3 * q + 9] = m1.x, d[3 * q + 11] = m1.y;
        d[3 * q + 18] = m2.x, d[3 * q + 20] = m2.y;
        inv3_t<L, DEFER>(d[3 * q + 1], d[3 * q + 10], d[3 * q + 19], uz, zc, z2);
    }
    // inverse along y: columns (p, r), the same pairs
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float2 m0 = make_float2(d[9 * r], d[9 * r + 2]), m1 = make_float2(d[9 * r + 3], d[9 * r + 5]),
               m2 = make_float2(d[9 * r + 6], d[9 * r + 8]);
        inv3_t<P, DEFER>(m0, m1, m2, P::splat(uy), P::splat(yc), P::splat(y2));
        d[9 * r] = m0.x, d[9 * r + 2] = m0.y, d[9 * r + 3] = m1.x, d[9 * r + 5] = m1.y;
        d[9 * r + 6] = m2.x, d[9 * r + 8] = m2.y;
        inv3_t<L, DEFER>(d[9 * r + 1], d[9 * r + 4], d[9 * r + 7], uy, yc, y2);
    }
    // inverse along x: rows, scalar
#pragma unroll
    for (int k = 0; k < 9; ++k) inv3_t<L, DEFER>(d[3 * k], d[3 * k + 1], d[3 * k + 2], ux, xc, x2);
}

template <bool DEFER = false>
__device__ __forceinline__ void collide_fast(float (&d)[Q], const LevelArgs& a)
{
    collide_fast_p<DEFER>(d, a.s2, a.g);
}

// The classical operators the paper compares against (Sec. 2.1.2), with the second-order
// equilibrium f_eq2_i = w_i rho [1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u] and the second-order (Guo)
// force term F_i = w_i [3 (c - u) + 9 (c.u) c] . F, F = rho g, u = j / rho + g / 2.
// TRT: the even and odd parts of each pair (i, opp(i)) relax with a.s2 and a.wm; the even and
// odd parts of F_i are scaled by (1 - s2/2) and (1 - wm/2).  SRT2 is the case wm = s2.
// Deviation form throughout: with d = f - w, f_eq2 - w = w [(rho - 1) + rho (3 c.u + 4.5 (c.u)^2
// - 1.5 u.u)], so the O(1) weights never enter a rounding.  The FP32 weights are not exact:
// sum_i w_i and sum_i 3 w_i c_i c_i differ from 1 and the identity by ~3e-8, so relaxing toward
// f_eq2 would create mass omega * 3e-8 * (rho - 1) and momentum omega * 3e-8 * rho u every step
// (a systematic drift that grows with time, unlike rounding).  The post-collision mass and
// momentum are therefore restored to their exact values rho and j + F: mass through the rest
// population, momentum through the three face pairs (each pair's difference carries one axis
// and leaves the mass unchanged).
template <bool TRT>
__device__ __forceinline__ void collide_trt2(float (&d)[Q], const LevelArgs& a)
{
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (cx_of(i)) jx += cx_of(i) > 0 ? d[i] : -d[i];
        if (cy_of(i)) jy += cy_of(i) > 0 ? d[i] : -d[i];
        if (cz_of(i)) jz += cz_of(i) > 0 ? d[i] : -d[i];
    }
    const float rho = 1.0f + drho, ir = 1.0f / rho;
    const float ux = fmaf(jx, ir, 0.5f * a.g[0]), uy = fmaf(jy, ir, 0.5f * a.g[1]), uz = fmaf(jz, ir, 0.5f * a.g[2]);
    const float Fx = rho * a.g[0], Fy = rho * a.g[1], Fz = rho * a.g[2];
    const float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float uF3 = 3.0f * (ux * Fx + uy * Fy + uz * Fz);
    const float wp = a.s2, wm = TRT ? a.wm : a.s2;
    const float kp = 1.0f - 0.5f * wp, km = 1.0f - 0.5f * wm;
    {  // rest population: even only
        constexpr float w = w_of(13);
        const float peq = w * (drho - rho * uu15);
        d[13] = d[13] - wp * (d[13] - peq) - kp * w * uF3;
    }
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        const int o = Q - 1 - i;
        const float w = w_of(i);
        const float cu = (float)cx_of(i) * ux + (float)cy_of(i) * uy + (float)cz_of(i) * uz;
        const float cF = (float)cx_of(i) * Fx + (float)cy_of(i) * Fy + (float)cz_of(i) * Fz;
        const float peq = w * (drho + rho * (4.5f * cu * cu - uu15));
        const float meq = w * rho * 3.0f * cu;
        const float Fe = w * (9.0f * cu * cF - uF3), Fo = w * 3.0f * cF;
        const float p = 0.5f * (d[i] + d[o]), m = 0.5f * (d[i] - d[o]);
        const float ev = kp * Fe - wp * (p - peq), od = km * Fo - wm * (m - meq);
        d[i] = d[i] + ev + od;
        d[o] = d[o] + ev - od;
    }
    float pm = 0.0f, px = 0.0f, py = 0.0f, pz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        pm += d[i];
        if (cx_of(i)) px += cx_of(i) > 0 ? d[i] : -d[i];
        if (cy_of(i)) py += cy_of(i) > 0 ? d[i] : -d[i];
        if (cz_of(i)) pz += cz_of(i) > 0 ? d[i] : -d[i];
    }
    // face pairs (-x, +x) = (12, 14), (-y, +y) = (10, 16), (-z, +z) = (4, 22)
    const float hx = 0.5f * ((jx + Fx) - px), hy = 0.5f * ((jy + Fy) - py), hz = 0.5f * ((jz + Fz) - pz);
    d[14] += hx;
    d[12] -= hx;
    d[16] += hy;
    d[10] -= hy;
    d[22] += hz;
    d[4] -= hz;
    d[13] += drho - pm;
}

// DEFER (the default rates only): d leaves with the factors 2^nnz(c_i), for Store::store_x
template <int COLL, bool DEFER = false>
__device__ __forceinline__ void collide_model(float (&d)[Q], const LevelArgs& a)
{
    static_assert(!DEFER || COLL == COLL_CHM_FAST, "deferred halving is a form of the fast collision");
    if (COLL == COLL_CHM_FAST) collide_fast<DEFER>(d, a);
    else if (COLL == COLL_CHM) collide(d, a);
    else collide_trt2<COLL == COLL_TRT2>(d, a);
}

// A cell's own second-order rate s2 (an absorbing layer): SRT2 relaxes both parities with it,
// TRT2 derives its odd rate from it through Lambda.
template <int COLL>
__device__ __forceinline__ void set_own_rate(LevelArgs& la, float s2)
{
    la.s2 = s2;
    if (COLL == COLL_SRT2) la.wm = s2;
    if (COLL == COLL_TRT2) la.wm = 1.0f / (la.magic / (1.0f / s2 - 0.5f) + 0.5f);
}

// ------------------------------------------------------------------------------ gather (read-only)
// Populations of level n of one fluid cell, for the export and diagnostics kernels.
template <int ST, int SCHEME>
__device__ __forceinline__ void gather(const DomainView& v, const void* src, uint32_t slot, uint32_t word,
                                       const LevelArgs& a, float (&d)[Q])
{
    const uint32_t wm = word & WORD_WALL_MASK;
    const uint32_t n = (uint32_t)v.n_slots;
    if (SCHEME == LBM_SCHEME_ESOTERIC) {
        uint32_t cs[8];
        corner_slots(v.nb8 + (slot / BRICK_CELLS) * 8, slot, cs);
        fetch_et<ST, false>(src, n, cs, wm, a.parity, d);
    } else {
        fetch_ab<ST>(src, n, v.nbr + (slot / BRICK_CELLS) * Q, slot, wm, d);
    }
    if (wm) wall_rules<ST, SCHEME>(v, src, slot, word, a, d);
}

// ------------------------------------------------------------------------------ kernels
// One fused update of the cell at `slot` (a lane of a warp that covers half of one brick; all
// 32 lanes must call it together: the neighbour row goes round by shuffle).
template <int ST, int SCHEME, int COLL, int PC = -1>
__device__ __forceinline__ void step_cell(const DomainView& v, const void* src, void* dst, const LevelArgs& a,
                                          uint32_t slot, uint32_t lane)
{
    constexpr bool X = COLL == COLL_CHM_FAST;  // deferred halving in the inverse transform
    const uint32_t brick = slot / BRICK_CELLS;
    const uint32_t word = __ldg(v.word + slot);
    // the cell's record, loaded beside its word rather than after it: a Bouzidi or open cell then
    // waits for one memory latency fewer before its link values (4 bytes per slot of traffic)
    const int32_t auxv = __ldg(v.aux + slot);
    const bool fluid = (word & WORD_FLUID) != 0u;
    const uint32_t wm = word & WORD_WALL_MASK;
    const uint32_t n = (uint32_t)v.n_slots;
    float d[Q];
    LevelArgs la = a;
    if (word & WORD_OWN_TAU) set_own_rate<COLL>(la, __ldg(v.s2_cell + slot));
    if (SCHEME == LBM_SCHEME_ESOTERIC) {
        const int32_t row = __ldg(v.nb8 + brick * 8u + (lane & 7u));
        uint32_t cs[8];
        corner_slots_shfl(row, slot, cs);
        const bool clean = PC >= 0 && __all_sync(0xffffffffu, wm == 0u);
        if (!fluid) return;
        fetch_et<ST, true, PC>(dst, n, cs, wm, a.parity, d, clean);
        const uint32_t half = wm ? wall_rules<ST, SCHEME>(v, nullptr, slot, word, a, d, auxv) : 0u;
        collide_model<COLL, X>(d, la);
        scale_out<ST, X>(d);
        store_et<ST, PC, X, true>(dst, n, cs, a.parity, d);
        if (half) {
            const uint32_t off = (uint32_t)auxv;
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((half & (1u << i)) && LBM_IN_RANGE(link_index(off, wm, i), v.n_bq, 5))
                    Store<ST>::store_h(v.side, link_index(off, wm, i), d[i]);
        }
    } else {
        const int32_t row = __ldg(v.nbr + brick * (uint32_t)Q + (lane < (uint32_t)Q ? lane : 0u));
        fetch_ab_shfl<ST>(src, n, row, slot, wm, fluid, d);
        if (!fluid) return;
        if (wm) wall_rules<ST, SCHEME>(v, src, slot, word, a, d, auxv);
        collide_model<COLL, X>(d, la);
        scale_out<ST, X>(d);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (!LBM_IN_RANGE((uint32_t)i * n + slot, (uint64_t)Q * n, 4)) continue;
            Store<ST>::store_h(dst, (uint32_t)i * n + slot, d[i]);
        }
    }
}

template <int ST, int SCHEME, int BRICKS, int MINB, int COLL, int PC = -1>
__global__ void __launch_bounds__(BRICKS * BRICK_CELLS, MINB)
    k_step(DomainView v, const void* src, void* dst, LevelArgs a)
{
    const uint32_t slot = blockIdx.x * (uint32_t)(BRICKS * BRICK_CELLS) + threadIdx.x;
    // the active slots are a multiple of 64, so this exit is taken by whole warps
    if (slot >= (uint32_t)(v.n_bricks * BRICK_CELLS)) return;
    step_cell<ST, SCHEME, COLL, PC>(v, src, dst, a, slot, threadIdx.x & 31u);
}

// Esoteric-twist step with two cells per thread: lane l of a warp updates cells l and l + 32 of
// one brick (its lower and upper halves along z), and their collisions run as one stream of packed
// FP32x2 instructions (the default rates only), which halves the issue slots of the arithmetic;
// loads, wall rules and stores stay per cell.  A warp covers one brick, so the brick's corner
// row still goes round by shuffle.  Results are bit-identical to the one-cell kernels.
template <int ST, int PC>
__device__ __forceinline__ void store_twist_cell(const DomainView& v, void* pop, const LevelArgs& a, uint32_t word,
                                                 int32_t aux, const uint32_t (&cs)[8], uint32_t half,
                                                 const float (&d)[Q])
{
    store_et<ST, PC, true, true>(pop, (uint32_t)v.n_slots, cs, a.parity, d);
    if (half) {
        const uint32_t off = (uint32_t)aux;
        const uint32_t wm = word & WORD_WALL_MASK;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if ((half & (1u << i)) && LBM_IN_RANGE(link_index(off, wm, i), v.n_bq, 5))
                Store<ST>::store_h(v.side, link_index(off, wm, i), d[i]);
    }
}

template <int ST, int BRICKS, int MINB, int PC>
__global__ void __launch_bounds__(BRICKS * 32, MINB)
    k_step2(DomainView v, void* pop, LevelArgs a)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t brick = blockIdx.x * (uint32_t)BRICKS + (threadIdx.x >> 5);
    if (brick >= (uint32_t)v.n_bricks) return;  // whole warps
    const uint32_t n = (uint32_t)v.n_slots;
    const uint32_t slotA = brick * BRICK_CELLS + lane, slotB = slotA + 32u;
    const int32_t row = __ldg(v.nb8 + brick * 8u + (lane & 7u));
    uint32_t csA[8], csB[8];
    corner_slots_shfl(row, slotA, csA);
    corner_slots_shfl(row, slotB, csB);
    const uint32_t wA = __ldg(v.word + slotA), wB = __ldg(v.word + slotB);
    const int32_t xA = __ldg(v.aux + slotA), xB = __ldg(v.aux + slotB);  // records, beside the words
    const bool fA = (wA & WORD_FLUID) != 0u, fB = (wB & WORD_FLUID) != 0u;
    const bool clean = PC >= 0 && __all_sync(0xffffffffu, ((wA | wB) & WORD_WALL_MASK) == 0u);
    if (!fA && !fB) return;
    float dA[Q], dB[Q];
    if (fA) fetch_et<ST, true, PC>(pop, n, csA, wA & WORD_WALL_MASK, a.parity, dA, clean);
    if (fB) fetch_et<ST, true, PC>(pop, n, csB, wB & WORD_WALL_MASK, a.parity, dB, clean);
    const uint32_t halfA =
        (fA && (wA & WORD_WALL_MASK)) ? wall_rules<ST, LBM_SCHEME_ESOTERIC>(v, nullptr, slotA, wA, a, dA, xA) : 0u;
    const uint32_t halfB =
        (fB && (wB & WORD_WALL_MASK)) ? wall_rules<ST, LBM_SCHEME_ESOTERIC>(v, nullptr, slotB, wB, a, dB, xB) : 0u;
    const float s2A = (wA & WORD_OWN_TAU) ? __ldg(v.s2_cell + slotA) : a.s2;
    const float s2B = (wB & WORD_OWN_TAU) ? __ldg(v.s2_cell + slotB) : a.s2;
    float2 d2[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d2[i] = make_float2(fA ? dA[i] : 0.0f, fB ? dB[i] : 0.0f);  // a solid lane: rest
    collide_fast_t<Lane2, true>(d2, make_float2(s2A, s2B), a.g);
    scale_out2<ST, true>(d2);  // the store factors of both cells, one packed multiply per direction
    if (fA) {
#pragma unroll
        for (int i = 0; i < Q; ++i) dA[i] = d2[i].x;
        store_twist_cell<ST, PC>(v, pop, a, wA, xA, csA, halfA, dA);
    }
    if (fB) {
#pragma unroll
        for (int i = 0; i < Q; ++i) dB[i] = d2[i].y;
        store_twist_cell<ST, PC>(v, pop, a, wB, xB, csB, halfB, dB);
    }
}

// Software-pipelined persistent variant of the FP32 esoteric-twist step.  Each CTA walks over
// chunks of BRICKS bricks; before computing chunk c, every thread issues cp.async copies of the
// 27 populations its cell of chunk c + gridDim will read (shared memory, one stage per chunk,
// two stages), so that the next cell's loads are in flight during the current cell's
// arithmetic without holding registers.  Each thread copies and reads only its own staging
// slots, so no CTA barrier is needed; and every location of the in-place array is owned by one
// cell, so prefetching another cell's locations before this cell's stores cannot race.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int BRICKS, int MINB, int COLL>
__global__ void __launch_bounds__(BRICKS * BRICK_CELLS, MINB)
    k_step_et_pipe(DomainView v, float* __restrict__ pop, LevelArgs a)
{
    constexpr int T = BRICKS * BRICK_CELLS;
    extern __shared__ float stage[];  // [2][27][T]
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t n = (uint32_t)v.n_slots;
    const int64_t n_chunks = (v.n_bricks + BRICKS - 1) / BRICKS;
    // issue the copies of chunk c into stage st (all lanes run the shuffles)
    auto prefetch = [&](int64_t c, int st) {
        const uint32_t slot = (uint32_t)(c * T) + tid;
        if (slot < (uint32_t)(v.n_bricks * BRICK_CELLS)) {
            const uint32_t word = __ldg(v.word + slot);
            const int32_t row = __ldg(v.nb8 + (slot / BRICK_CELLS) * 8u + (lane & 7u));
            uint32_t cs[8];
            corner_slots_shfl(row, slot, cs);
            if (word & WORD_FLUID) {
                const uint32_t wm = word & WORD_WALL_MASK;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const uint32_t flip = ((uint32_t)a.parity ^ (wm >> i)) & 1u;
                    const uint32_t dir = flip ? (uint32_t)(Q - 1 - i) : (uint32_t)i;
                    if (LBM_IN_RANGE(dir * n + cs[corner_neg(i)], (uint64_t)Q * n, 2))
                        cp_async4(&stage[(st * Q + i) * T + tid], pop + dir * n + cs[corner_neg(i)]);
                }
            }
        }
        cp_async_commit();
    };
    int st = 0;
    int64_t c = blockIdx.x;
    if (c < n_chunks) prefetch(c, 0);
    for (; c < n_chunks; c += gridDim.x) {
        prefetch(c + gridDim.x, st ^ 1);  // an empty group past the end keeps the count aligned
        cp_async_wait_one();
        const uint32_t slot = (uint32_t)(c * T) + tid;
        if (slot < (uint32_t)(v.n_bricks * BRICK_CELLS)) {
            const uint32_t word = __ldg(v.word + slot);
            const int32_t row = __ldg(v.nb8 + (slot / BRICK_CELLS) * 8u + (lane & 7u));
            uint32_t cs[8];
            corner_slots_shfl(row, slot, cs);
            if (word & WORD_FLUID) {
                const uint32_t wm = word & WORD_WALL_MASK;
                LevelArgs la = a;
                if (word & WORD_OWN_TAU) set_own_rate<COLL>(la, __ldg(v.s2_cell + slot));
                float d[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) d[i] = stage[(st * Q + i) * T + tid];
                const uint32_t half = wm ? wall_rules<LBM_STORE_FP32, LBM_SCHEME_ESOTERIC>(v, nullptr, slot, word, a, d) : 0u;
                collide_model<COLL>(d, la);
                store_et<LBM_STORE_FP32>(pop, n, cs, a.parity, d);
                if (half) {
                    const uint32_t off = (uint32_t)v.aux[slot];
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if ((half & (1u << i)) && LBM_IN_RANGE(link_index(off, wm, i), v.n_bq, 5))
                            Store<LBM_STORE_FP32>::store(v.side, i, link_index(off, wm, i), d[i]);
                }
            }
        }
        st ^= 1;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Several domains (esoteric twist, one storage precision) in one launch: the CTAs run over the
// concatenated brick lists; each warp finds its domain by binary search in the brick prefix
// sums and updates one of that domain's half-bricks with the domain's own level arguments.
template <int ST, int BRICKS, int MINB, int COLL, int PC = -1>
__global__ void __launch_bounds__(BRICKS * BRICK_CELLS, MINB)
    k_step_batch(const BatchEntry* __restrict__ ent, const int64_t* __restrict__ brick_start, int n_dom,
                 const LevelArgs* __restrict__ args)
{
    const int64_t gslot = (int64_t)blockIdx.x * (BRICKS * BRICK_CELLS) + threadIdx.x;
    const int64_t gbrick = gslot / BRICK_CELLS;
    if (gbrick >= __ldg(brick_start + n_dom)) return;  // whole warps
    int lo = 0, hi = n_dom - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(brick_start + mid) <= gbrick) lo = mid;
        else hi = mid - 1;
    }
    const DomainView v = ent[lo].view;
    const LevelArgs a = args[lo];
    const uint32_t slot = (uint32_t)((gbrick - __ldg(brick_start + lo)) * BRICK_CELLS) + (threadIdx.x & 63u);
    step_cell<ST, LBM_SCHEME_ESOTERIC, COLL, PC>(v, ent[lo].pop, ent[lo].pop, a, slot, threadIdx.x & 31u);
}

// Persistent form of the batched step: one launch advances every domain `steps` steps.  The CTAs
// (all resident: the launch is cooperative) stride over the concatenated brick list, BRICKS bricks
// per unit of work, and meet at a grid-wide barrier after each step, since the twist's next step
// reads what neighbouring CTAs wrote.  Every wait at the barrier is bounded by `limit_ns` of the
// global timer: a CTA that gives up raises bar->fail and every CTA leaves at its next barrier, so
// a chunk that cannot complete ends instead of hanging (the host then reports LBM_ERR_TIMEOUT).
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true when every CTA has finished step s; false when this CTA or another gave up
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned int target, uint64_t limit_ns)
{
    __shared__ int ok;
    __syncthreads();  // this CTA's writes of the step are done
    if (threadIdx.x == 0) {
        int good = 1;
        __threadfence();  // release them at GPU scope before arriving
        atomicAdd(&bar->count, 1u);
        const uint64_t t0 = global_ns();
        while (true) {
            unsigned int c, f;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(&bar->count) : "memory");
            if (c >= target) break;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(&bar->fail) : "memory");
            if (f) {
                good = 0;
                break;
            }
            if (global_ns() - t0 > limit_ns) {
                atomicExch(&bar->fail, 1u);
                good = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

template <int ST, int BRICKS, int MINB, int COLL, int P0>
__global__ void __launch_bounds__(BRICKS * BRICK_CELLS, MINB)
    k_step_batch_persistent(const BatchEntry* __restrict__ ent, const int64_t* __restrict__ brick_start, int n_dom,
                            const LevelArgs* __restrict__ args, int steps, GridBarrier* bar, unsigned int* tickets,
                            uint64_t limit_ns)
{
    const int64_t total = __ldg(brick_start + n_dom);
    const int64_t n_units = (total + BRICKS - 1) / BRICKS;
    __shared__ unsigned int next;
    for (int s = 0; s < steps; ++s) {
        // units of step s are handed out by a ticket counter (tickets[s], cleared before the
        // launch), so that CTAs that finish early take more
        for (;;) {
            __syncthreads();  // every thread has read the previous ticket
            if (threadIdx.x == 0) next = atomicAdd(&tickets[s], 1u);
            __syncthreads();
            const int64_t unit = next;
            if (unit >= n_units) break;
            const int64_t gbrick = unit * BRICKS + (threadIdx.x / BRICK_CELLS);
            if (gbrick < total) {  // whole warps
                int lo = 0, hi = n_dom - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(brick_start + mid) <= gbrick) lo = mid;
                    else hi = mid - 1;
                }
                const DomainView v = ent[lo].view;
                const LevelArgs a = args[(size_t)s * n_dom + lo];
                const uint32_t slot =
                    (uint32_t)((gbrick - __ldg(brick_start + lo)) * BRICK_CELLS) + (threadIdx.x & 63u);
                // P0 >= 0: every member has parity P0 at step 0, so step s has parity P0 ^ (s & 1)
                if (P0 >= 0 && ((s & 1) ^ P0) == 0)
                    step_cell<ST, LBM_SCHEME_ESOTERIC, COLL, (P0 >= 0 ? 0 : -1)>(v, ent[lo].pop, ent[lo].pop, a, slot,
                                                                                 threadIdx.x & 31u);
                else if (P0 >= 0)
                    step_cell<ST, LBM_SCHEME_ESOTERIC, COLL, (P0 >= 0 ? 1 : -1)>(v, ent[lo].pop, ent[lo].pop, a, slot,
                                                                                 threadIdx.x & 31u);
                else
                    step_cell<ST, LBM_SCHEME_ESOTERIC, COLL, -1>(v, ent[lo].pop, ent[lo].pop, a, slot, threadIdx.x & 31u);
            }
        }
        if (s + 1 < steps && !grid_barrier(bar, (unsigned int)(s + 1) * gridDim.x, limit_ns)) return;
    }
}

// Running means (the time averaging of Sec. 3.3): sums[k] += (rho, ux, uy, uz) of fluid cell k at
// the current level, in FP64 so that thousands of samples add without loss.
template <int ST, int SCHEME>
__global__ void __launch_bounds__(256)
    k_mean_sample(DomainView v, const void* src, LevelArgs a, const int32_t* fl_slot, int64_t n_fluid, Sum4* sums)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_fluid) return;
    const uint32_t slot = (uint32_t)fl_slot[k];
    float d[Q];
    gather<ST, SCHEME>(v, src, slot, v.word[slot], a, d);
    const Moments M = moments(d, a.g);
    Sum4 s = sums[k];
    s.x += (double)M.rho;
    s.y += (double)M.ux;
    s.z += (double)M.uy;
    s.w += (double)M.uz;
    sums[k] = s;
}

// Monitoring-point probes (Sec. 2.2.2 follows the velocity at points around the sac):
// out[p] = (rho, ux, uy, uz) of fluid cell idx[p] (fluid index: box order, x fastest); an index
// outside [0, n_fluid) gives NaNs.
template <int ST, int SCHEME>
__global__ void __launch_bounds__(128)
    k_probe(DomainView v, const void* src, LevelArgs a, const int32_t* fl_slot, int64_t n_fluid, const int64_t* idx,
            int n, float4* out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t k = idx[p];
    if (k < 0 || k >= n_fluid) {
        out[p] = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                             __int_as_float(0x7fc00000));
        return;
    }
    const uint32_t slot = (uint32_t)fl_slot[k];
    float d[Q];
    gather<ST, SCHEME>(v, src, slot, v.word[slot], a, d);
    const Moments M = moments(d, a.g);
    out[p] = make_float4(M.rho, M.ux, M.uy, M.uz);
}

template <int ST, int SCHEME>
__global__ void __launch_bounds__(256)
    k_macroscopic(DomainView v, const void* src, LevelArgs a, const int32_t* fl_slot, const int32_t* fl_box,
                  int64_t n_fluid, int dense, float* rho, float* u, int64_t n_out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_fluid) return;
    const uint32_t slot = (uint32_t)fl_slot[k];
    float d[Q];
    gather<ST, SCHEME>(v, src, slot, v.word[slot], a, d);
    const Moments M = moments(d, a.g);
    const int64_t o = dense ? (int64_t)fl_box[k] : k;
    rho[o] = M.rho;
    u[o] = M.ux;
    u[n_out + o] = M.uy;
    u[2 * n_out + o] = M.uz;
}

// Post-collision populations of the previous level := f_eq(rho, u) (full expansion, product
// form), written as deviations d_i = rho (prod psi - w_i) + (rho - 1) w_i with
// prod psi - w = dpx psi_y psi_z + w1x dpy psi_z + w1x w1y dpz, dpsi(0) = -u^2,
// dpsi(+-1) = (+-u + u^2)/2.  A-B: into the cell's own slots; twist: where the step of parity
// `parity_prev` would have written them, plus every direction into the side buffer of a
// Bouzidi cell.
template <int ST, int SCHEME>
__global__ void __launch_bounds__(256)
    k_init_equilibrium(DomainView v, void* dst, int parity_prev, const int32_t* fl_slot, const int32_t* fl_box,
                       int64_t n_fluid, const float* rho_in, const float* u_in, int64_t n_box)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_fluid) return;
    const int64_t b = fl_box[k];
    const uint32_t slot = (uint32_t)fl_slot[k];
    const float rho = rho_in[b];
    const float u[3] = {u_in[b], u_in[n_box + b], u_in[2 * n_box + b]};
    float dp[3][3], ps[3][3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float uu = u[ax] * u[ax];
        dp[ax][0] = 0.5f * (uu - u[ax]);
        dp[ax][1] = -uu;
        dp[ax][2] = 0.5f * (uu + u[ax]);
        ps[ax][0] = 1.0f / 6.0f + dp[ax][0];
        ps[ax][1] = 2.0f / 3.0f + dp[ax][1];
        ps[ax][2] = 1.0f / 6.0f + dp[ax][2];
    }
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ix = cx_of(i) + 1, iy = cy_of(i) + 1, iz = cz_of(i) + 1;
        const float w1x = w1_of(cx_of(i)), w1y = w1_of(cy_of(i));
        const float dprod = dp[0][ix] * ps[1][iy] * ps[2][iz] + w1x * dp[1][iy] * ps[2][iz] + w1x * w1y * dp[2][iz];
        d[i] = fmaf(rho, dprod, (rho - 1.0f) * w_of(i));
    }
    const uint32_t n = (uint32_t)v.n_slots;
    if (SCHEME == LBM_SCHEME_ESOTERIC) {
        uint32_t cs[8];
        corner_slots(v.nb8 + (slot / BRICK_CELLS) * 8, slot, cs);
        store_et<ST>(dst, n, cs, parity_prev, d);
        const uint32_t word = v.word[slot];
        if (((word >> WORD_KIND_SHIFT) & 3u) == KIND_BOUZIDI) {
            const uint32_t off = (uint32_t)v.aux[slot];
            const uint32_t wm = word & WORD_WALL_MASK;
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (((wm >> i) & 1u) && LBM_IN_RANGE(link_index(off, wm, i), v.n_bq, 5))
                    Store<ST>::store(v.side, i, link_index(off, wm, i), d[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (LBM_IN_RANGE((uint32_t)i * n + slot, (uint64_t)Q * n, 4)) Store<ST>::store(dst, i, (uint32_t)i * n + slot, d[i]);
    }
}

// Velocity correction (learned corrector): the post-collision populations of the previous level
// gain rho (prod psi(u + du) - prod psi(u)) at every fluid cell except inlet and outlet cells,
// rho and u those of the current level.  The product difference is expanded, (a + da)(b + db)(c + dc) - abc =
// da (b + db)(c + dc) + a db (c + dc) + a b dc, with dpsi(0) = -(2u + du) du and
// dpsi(+-1) = (+-du + (2u + du) du)/2, so that no O(1) value is rounded against a small one.
template <int ST, int SCHEME>
__global__ void __launch_bounds__(256)
    k_apply_du(DomainView v, void* pop, int parity_prev, const int32_t* fl_slot, const int32_t* fl_box, int64_t n_fluid,
               const float* rho_in, const float* u_in, const float* du_in, int64_t n_box)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_fluid) return;
    const int64_t b = fl_box[k];
    const uint32_t slot = (uint32_t)fl_slot[k];
    // open-boundary cells are left alone: their closures rebuild the unknowns every step
    const uint32_t word = v.word[slot];
    if (((word >> WORD_KIND_SHIFT) & 3u) >= KIND_INLET) return;
    const float rho = rho_in[b];
    float ps[3][3], dp[3][3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float u = u_in[ax * n_box + b], du = du_in[ax * n_box + b];
        const float uu = u * u;
        ps[ax][0] = 1.0f / 6.0f + 0.5f * (uu - u);
        ps[ax][1] = 2.0f / 3.0f - uu;
        ps[ax][2] = 1.0f / 6.0f + 0.5f * (uu + u);
        const float s2 = (2.0f * u + du) * du;
        dp[ax][0] = 0.5f * (s2 - du);
        dp[ax][1] = -s2;
        dp[ax][2] = 0.5f * (s2 + du);
    }
    float delta[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ix = cx_of(i) + 1, iy = cy_of(i) + 1, iz = cz_of(i) + 1;
        const float by = ps[1][iy] + dp[1][iy], bz = ps[2][iz] + dp[2][iz];
        delta[i] = rho * (dp[0][ix] * by * bz + ps[0][ix] * dp[1][iy] * bz + ps[0][ix] * ps[1][iy] * dp[2][iz]);
    }
    // every read is issued before the first write: the compiler cannot tell that a write does not
    // alias the next read, so read-modify-write pairs in one loop would wait for one memory
    // latency each
    const uint32_t n = (uint32_t)v.n_slots;
    uint32_t off[Q];
    float f[Q];
    if (SCHEME == LBM_SCHEME_ESOTERIC) {
        uint32_t cs[8];
        corner_slots(v.nb8 + (slot / BRICK_CELLS) * 8, slot, cs);
#pragma unroll
        for (int i = 0; i < Q; ++i) off[i] = (parity_prev ? (uint32_t)i : (uint32_t)(Q - 1 - i)) * n + cs[corner_pos(i)];
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) off[i] = (uint32_t)i * n + slot;
    }
    const bool bouzidi = SCHEME == LBM_SCHEME_ESOTERIC && ((word >> WORD_KIND_SHIFT) & 3u) == KIND_BOUZIDI;
    const uint32_t wm = bouzidi ? (word & WORD_WALL_MASK) : 0u;
    const uint32_t off0 = bouzidi ? (uint32_t)v.aux[slot] : 0u;
    float fs[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = LBM_IN_RANGE(off[i], (uint64_t)Q * n, 7) ? Store<ST>::load_rw(pop, i, off[i]) : 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        fs[i] = (((wm >> i) & 1u) && LBM_IN_RANGE(link_index(off0, wm, i), v.n_bq, 5))
                    ? Store<ST>::load_rw(v.side, i, link_index(off0, wm, i))
                    : 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (LBM_IN_RANGE(off[i], (uint64_t)Q * n, 7)) Store<ST>::store(pop, i, off[i], f[i] + delta[i]);
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (((wm >> i) & 1u) && LBM_IN_RANGE(link_index(off0, wm, i), v.n_bq, 5))
            Store<ST>::store(v.side, i, link_index(off0, wm, i), fs[i] + delta[i]);
}

// FP64 diagnostics: per-block partial sums in a fixed order; one block then reduces the
// partials in a fixed order (reproducible run to run).
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_FIELDS = 5;  // mass, flux_in, flux_out, max|u|, non-finite count

__device__ __forceinline__ void block_reduce5(double (&x)[DIAG_FIELDS], double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int f = 0; f < DIAG_FIELDS; ++f) {
            const double o = __shfl_down_sync(0xffffffffu, x[f], off);
            x[f] = (f == 3) ? fmax(x[f], o) : x[f] + o;
        }
    }
    if (lane == 0)
        for (int f = 0; f < DIAG_FIELDS; ++f) sh[warp * DIAG_FIELDS + f] = x[f];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < DIAG_THREADS / 32; ++w)
            for (int f = 0; f < DIAG_FIELDS; ++f)
                x[f] = (f == 3) ? fmax(x[f], sh[w * DIAG_FIELDS + f]) : x[f] + sh[w * DIAG_FIELDS + f];
    }
}

template <int ST, int SCHEME>
__global__ void __launch_bounds__(DIAG_THREADS)
    k_diagnostics(DomainView v, const void* src, LevelArgs a, const int32_t* fl_slot, int64_t n_fluid,
                  double* partials)
{
    __shared__ double sh[(DIAG_THREADS / 32) * DIAG_FIELDS];
    double x[DIAG_FIELDS] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t k = (int64_t)blockIdx.x * DIAG_THREADS + threadIdx.x;
    if (k < n_fluid) {
        const uint32_t slot = (uint32_t)fl_slot[k];
        const uint32_t word = v.word[slot];
        float d[Q];
        gather<ST, SCHEME>(v, src, slot, word, a, d);
        const Moments M = moments(d, a.g);
        const bool finite = isfinite(M.rho) && isfinite(M.ux) && isfinite(M.uy) && isfinite(M.uz);
        if (finite) {
            x[0] = (double)M.rho;
            const int kind = (int)((word >> WORD_KIND_SHIFT) & 3u);
            if (kind >= KIND_INLET && LBM_IN_RANGE(v.aux[slot], v.n_io, 6)) {
                const int64_t rec = v.aux[slot];
                const int ax = v.io_axis[rec];
                const float un = v.io_sign[rec] * (ax == 0 ? M.ux : ax == 1 ? M.uy : M.uz);
                if (kind == KIND_INLET) x[1] = (double)M.rho * (double)un;
                else x[2] = -(double)M.rho * (double)un;
            }
            x[3] = sqrt((double)M.ux * M.ux + (double)M.uy * M.uy + (double)M.uz * M.uz);
        } else {
            x[4] = 1.0;
        }
    }
    block_reduce5(x, sh);
    if (threadIdx.x == 0)
        for (int f = 0; f < DIAG_FIELDS; ++f) partials[(int64_t)blockIdx.x * DIAG_FIELDS + f] = x[f];
}

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

// Calls f(std::integral_constant<int, COLL>{}) for the collision kernel `coll`.
template <class F>
cudaError_t with_coll(int coll, F&& f)
{
    switch (coll) {
    case COLL_CHM: return f(std::integral_constant<int, COLL_CHM>{});
    case COLL_CHM_FAST: return f(std::integral_constant<int, COLL_CHM_FAST>{});
    case COLL_SRT2: return f(std::integral_constant<int, COLL_SRT2>{});
    default: return f(std::integral_constant<int, COLL_TRT2>{});
    }
}

// ------------------------------------------------------------------------------ launchers
// Launch configurations of the step kernel: (bricks per CTA, minimum resident CTAs per SM);
// the second number sets the register budget, 65536 / (threads * CTAs).
template <int ST, int SCHEME, int BRICKS, int MINB>
cudaError_t launch_step_t(const DomainView& v, const void* src, void* dst, const LevelArgs& a, cudaStream_t s)
{
    if (v.n_bricks == 0) return cudaSuccess;
    const int grid = grid_for(v.n_bricks, BRICKS);
    return with_coll(a.coll, [&](auto c) {
        constexpr int C = decltype(c)::value;
        // the twist with the default rates has one kernel per parity (constant plane indices)
        if constexpr (SCHEME == LBM_SCHEME_ESOTERIC && C == COLL_CHM_FAST) {
            if (a.parity) k_step<ST, SCHEME, BRICKS, MINB, C, 1><<<grid, BRICKS * BRICK_CELLS, 0, s>>>(v, src, dst, a);
            else k_step<ST, SCHEME, BRICKS, MINB, C, 0><<<grid, BRICKS * BRICK_CELLS, 0, s>>>(v, src, dst, a);
        } else {
            k_step<ST, SCHEME, BRICKS, MINB, C><<<grid, BRICKS * BRICK_CELLS, 0, s>>>(v, src, dst, a);
        }
        return cudaGetLastError();
    });
}

template <int ST, int BRICKS, int MINB>
cudaError_t launch_step2(const DomainView& v, void* pop, const LevelArgs& a, cudaStream_t s)
{
    if (v.n_bricks == 0) return cudaSuccess;
    // runtime parity: the constant-plane form of the one-cell kernels was slower here (the two
    // cells' addresses compete with the packed collision for the 128-register budget)
    k_step2<ST, BRICKS, MINB, -1><<<grid_for(v.n_bricks, BRICKS), BRICKS * 32, 0, s>>>(v, pop, a);
    return cudaGetLastError();
}

template <int BRICKS, int MINB>
cudaError_t launch_step_et_pipe(const DomainView& v, void* pop, const LevelArgs& a, cudaStream_t s)
{
    if (v.n_bricks == 0) return cudaSuccess;
    constexpr int T = BRICKS * BRICK_CELLS;
    const size_t smem = sizeof(float) * 2 * Q * T;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n_chunks = (v.n_bricks + BRICKS - 1) / BRICKS;
    const int grid = (int)std::min<int64_t>(n_chunks, (int64_t)sms * MINB);
    return with_coll(a.coll, [&](auto c) {
        auto k = k_step_et_pipe<BRICKS, MINB, decltype(c)::value>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, T, smem, s>>>(v, static_cast<float*>(pop), a);
        return cudaGetLastError();
    });
}

template <int ST, int SCHEME>
cudaError_t launch_step_scheme(int config, const DomainView& v, const void* src, void* dst, const LevelArgs& a,
                               cudaStream_t s)
{
    if (config == 5) {
        if (ST == LBM_STORE_FP32 && SCHEME == LBM_SCHEME_ESOTERIC) return launch_step_et_pipe<2, 6>(v, dst, a, s);
        config = 3;  // the pipelined variant exists for FP32 twist only
    }
    if (config >= 6) {
        if (SCHEME == LBM_SCHEME_ESOTERIC && a.coll == COLL_CHM_FAST)
            return config == 6 ? launch_step2<ST, 4, 4>(v, dst, a, s) : launch_step2<ST, 4, 3>(v, dst, a, s);
        config = 2;  // the two-cell kernels exist for the twist with the default rates only
    }
    switch (config) {
    case 0: return launch_step_t<ST, SCHEME, 4, 3>(v, src, dst, a, s);
    case 1: return launch_step_t<ST, SCHEME, 2, 7>(v, src, dst, a, s);
    case 2: return launch_step_t<ST, SCHEME, 2, 6>(v, src, dst, a, s);
    case 3: return launch_step_t<ST, SCHEME, 2, 8>(v, src, dst, a, s);
    default: return launch_step_t<ST, SCHEME, 2, 10>(v, src, dst, a, s);
    }
}

template <int ST>
cudaError_t launch_step(int scheme, int config, const DomainView& v, const void* src, void* dst,
                        const LevelArgs& a, cudaStream_t s)
{
    return scheme == LBM_SCHEME_ESOTERIC ? launch_step_scheme<ST, LBM_SCHEME_ESOTERIC>(config, v, src, dst, a, s)
                                         : launch_step_scheme<ST, LBM_SCHEME_AB>(config, v, src, dst, a, s);
}

// the export and the correction run one thread per fluid cell; with small CTAs a domain of a few
// ten thousand cells still spreads over every SM (its latency chains overlap on all of them)
constexpr int PER_CELL_THREADS = 64;

template <int ST>
cudaError_t launch_macroscopic(int scheme, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, const int32_t* fl_box, int64_t n_fluid, int dense, float* rho,
                               float* u, int64_t n_out, cudaStream_t s)
{
    if (n_fluid == 0) return cudaSuccess;
    if (scheme == LBM_SCHEME_ESOTERIC)
        k_macroscopic<ST, LBM_SCHEME_ESOTERIC><<<grid_for(n_fluid, PER_CELL_THREADS), PER_CELL_THREADS, 0, s>>>(v, src, a, fl_slot, fl_box,
                                                                                  n_fluid, dense, rho, u, n_out);
    else
        k_macroscopic<ST, LBM_SCHEME_AB><<<grid_for(n_fluid, PER_CELL_THREADS), PER_CELL_THREADS, 0, s>>>(v, src, a, fl_slot, fl_box, n_fluid,
                                                                            dense, rho, u, n_out);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_mean_sample(int scheme, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, int64_t n_fluid, Sum4* sums, cudaStream_t s)
{
    if (n_fluid == 0) return cudaSuccess;
    if (scheme == LBM_SCHEME_ESOTERIC)
        k_mean_sample<ST, LBM_SCHEME_ESOTERIC><<<grid_for(n_fluid, 256), 256, 0, s>>>(v, src, a, fl_slot, n_fluid, sums);
    else
        k_mean_sample<ST, LBM_SCHEME_AB><<<grid_for(n_fluid, 256), 256, 0, s>>>(v, src, a, fl_slot, n_fluid, sums);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_probe(int scheme, const DomainView& v, const void* src, const LevelArgs& a, const int32_t* fl_slot,
                         int64_t n_fluid, const int64_t* idx, int n, float4* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (scheme == LBM_SCHEME_ESOTERIC)
        k_probe<ST, LBM_SCHEME_ESOTERIC><<<grid_for(n, 128), 128, 0, s>>>(v, src, a, fl_slot, n_fluid, idx, n, out);
    else
        k_probe<ST, LBM_SCHEME_AB><<<grid_for(n, 128), 128, 0, s>>>(v, src, a, fl_slot, n_fluid, idx, n, out);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_init_equilibrium(int scheme, const DomainView& v, void* dst, int parity_prev,
                                    const int32_t* fl_slot, const int32_t* fl_box, int64_t n_fluid,
                                    const float* rho, const float* u, int64_t n_box, cudaStream_t s)
{
    if (n_fluid == 0) return cudaSuccess;
    if (scheme == LBM_SCHEME_ESOTERIC)
        k_init_equilibrium<ST, LBM_SCHEME_ESOTERIC><<<grid_for(n_fluid, 256), 256, 0, s>>>(
            v, dst, parity_prev, fl_slot, fl_box, n_fluid, rho, u, n_box);
    else
        k_init_equilibrium<ST, LBM_SCHEME_AB><<<grid_for(n_fluid, 256), 256, 0, s>>>(
            v, dst, parity_prev, fl_slot, fl_box, n_fluid, rho, u, n_box);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_diagnostics(int scheme, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, int64_t n_fluid, double* partials, cudaStream_t s)
{
    const int nb = (int)diagnostics_blocks(n_fluid);
    if (scheme == LBM_SCHEME_ESOTERIC)
        k_diagnostics<ST, LBM_SCHEME_ESOTERIC><<<nb, DIAG_THREADS, 0, s>>>(v, src, a, fl_slot, n_fluid, partials);
    else
        k_diagnostics<ST, LBM_SCHEME_AB><<<nb, DIAG_THREADS, 0, s>>>(v, src, a, fl_slot, n_fluid, partials);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_apply_du(int scheme, const DomainView& v, void* pop, int parity_prev, const int32_t* fl_slot,
                           const int32_t* fl_box, int64_t n_fluid, const float* rho, const float* u, const float* du,
                           int64_t n_box, cudaStream_t s)
{
    if (n_fluid == 0) return cudaSuccess;
    if (scheme == LBM_SCHEME_ESOTERIC)
        k_apply_du<ST, LBM_SCHEME_ESOTERIC><<<grid_for(n_fluid, PER_CELL_THREADS), PER_CELL_THREADS, 0, s>>>(v, pop, parity_prev, fl_slot, fl_box,
                                                                               n_fluid, rho, u, du, n_box);
    else
        k_apply_du<ST, LBM_SCHEME_AB><<<grid_for(n_fluid, PER_CELL_THREADS), PER_CELL_THREADS, 0, s>>>(v, pop, parity_prev, fl_slot, fl_box, n_fluid,
                                                                         rho, u, du, n_box);
    return cudaGetLastError();
}

template <int ST, int BRICKS, int MINB>
cudaError_t launch_step_batch_t(const BatchEntry* ent, const int64_t* brick_start, int n_dom, int64_t total_bricks,
                                const LevelArgs* args, int coll, int parity, cudaStream_t s)
{
    if (total_bricks == 0) return cudaSuccess;
    const int grid = grid_for(total_bricks, BRICKS);
    return with_coll(coll, [&](auto c) {
        constexpr int C = decltype(c)::value;
        // one kernel per parity when every domain has the same one (constant plane indices)
        if constexpr (C == COLL_CHM_FAST) {
            if (parity == 0)
                k_step_batch<ST, BRICKS, MINB, C, 0><<<grid, BRICKS * BRICK_CELLS, 0, s>>>(ent, brick_start, n_dom, args);
            else if (parity == 1)
                k_step_batch<ST, BRICKS, MINB, C, 1><<<grid, BRICKS * BRICK_CELLS, 0, s>>>(ent, brick_start, n_dom, args);
            else
                k_step_batch<ST, BRICKS, MINB, C><<<grid, BRICKS * BRICK_CELLS, 0, s>>>(ent, brick_start, n_dom, args);
        } else {
            k_step_batch<ST, BRICKS, MINB, C><<<grid, BRICKS * BRICK_CELLS, 0, s>>>(ent, brick_start, n_dom, args);
        }
        return cudaGetLastError();
    });
}

// one cooperative launch of k_step_batch_persistent (128 threads, 8 CTAs per SM at most): as many
// CTAs as can be resident, never more than units of work; bar is followed by `steps` ticket
// counters, all cleared before the launch
template <int ST, int COLL, int P0>
cudaError_t launch_persistent_t(const BatchEntry* ent, const int64_t* brick_start, int n_dom, int64_t total_bricks,
                                const LevelArgs* args, int steps, GridBarrier* bar, uint64_t limit_ns, cudaStream_t s)
{
    constexpr int BRICKS = 2, MINB = 8;
    unsigned int* tickets = reinterpret_cast<unsigned int*>(bar + 1);  // [steps] after the barrier word
    auto k = k_step_batch_persistent<ST, BRICKS, MINB, COLL, P0>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BRICKS * BRICK_CELLS, 0);
    if (e != cudaSuccess) return e;
    const int64_t units = (total_bricks + BRICKS - 1) / BRICKS;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)sms * per_sm));
    void* kargs[] = {(void*)&ent, (void*)&brick_start, (void*)&n_dom, (void*)&args, (void*)&steps, (void*)&bar,
                     (void*)&tickets, (void*)&limit_ns};
    return cudaLaunchCooperativeKernel((const void*)k, dim3(grid), dim3(BRICKS * BRICK_CELLS), kargs, 0, s);
}

template <int ST>
cudaError_t launch_step_batch_persistent(const BatchEntry* ent, const int64_t* brick_start, int n_dom,
                                         int64_t total_bricks, const LevelArgs* args, int coll, int parity0, int steps,
                                         GridBarrier* bar, uint64_t limit_ns, cudaStream_t s)
{
    if (total_bricks == 0 || steps == 0) return cudaSuccess;
    return with_coll(coll, [&](auto c) {
        constexpr int C = decltype(c)::value;
        // parity-specialised steps for the default rates when the members share a parity
        if constexpr (C == COLL_CHM_FAST) {
            if (parity0 == 0)
                return launch_persistent_t<ST, C, 0>(ent, brick_start, n_dom, total_bricks, args, steps, bar, limit_ns, s);
            if (parity0 == 1)
                return launch_persistent_t<ST, C, 1>(ent, brick_start, n_dom, total_bricks, args, steps, bar, limit_ns, s);
        }
        return launch_persistent_t<ST, C, -1>(ent, brick_start, n_dom, total_bricks, args, steps, bar, limit_ns, s);
    });
}

template <int ST>
cudaError_t launch_step_batch(int config, const BatchEntry* ent, const int64_t* brick_start, int n_dom,
                              int64_t total_bricks, const LevelArgs* args, int coll, int parity, cudaStream_t s)
{
    switch (config) {
    case 0: return launch_step_batch_t<ST, 4, 3>(ent, brick_start, n_dom, total_bricks, args, coll, parity, s);
    case 1: return launch_step_batch_t<ST, 2, 7>(ent, brick_start, n_dom, total_bricks, args, coll, parity, s);
    case 2: return launch_step_batch_t<ST, 2, 6>(ent, brick_start, n_dom, total_bricks, args, coll, parity, s);
    case 3: return launch_step_batch_t<ST, 2, 8>(ent, brick_start, n_dom, total_bricks, args, coll, parity, s);
    default: return launch_step_batch_t<ST, 2, 10>(ent, brick_start, n_dom, total_bricks, args, coll, parity, s);
    }
}

// LBM_DEBUG: the first failed check's code since the last read (0: none), cleared on read; 0
// always in the default build
inline unsigned debug_fault()
{
#ifdef LBM_DEBUG
    unsigned h = 0u;
    const unsigned zero = 0u;
    if (cudaMemcpyFromSymbol(&h, g_debug_fault, sizeof(h)) != cudaSuccess) return 0xffffffffu;
    if (h) cudaMemcpyToSymbol(g_debug_fault, &zero, sizeof(zero));
    return h;
#else
    return 0u;
#endif
}

template <int ST>
const Launchers& make_launchers()
{
    static const Launchers L = {&launch_step<ST>,        &launch_macroscopic<ST>, &launch_init_equilibrium<ST>,
                                &launch_diagnostics<ST>, &launch_step_batch<ST>, &launch_apply_du<ST>,
                                &launch_mean_sample<ST>, &launch_probe<ST>,       &debug_fault,
                                &launch_step_batch_persistent<ST>};
    return L;
}

}  // namespace dev
}  // namespace lbm
