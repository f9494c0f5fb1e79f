// lbm_kernels.cu -- fused pull-stream / CHM-MRT collide kernel and its companions (export,
// equilibrium initialisation, FP64 diagnostics) for sm_103a.
//
// Method (Hosseini et al.):
//   LBE f_i(x + c_i, n + 1) = f_i(x, n) + Omega_i             (Sec. 2.1.1, first equation)
//   Omega = T^-1 S T (f_eq - f), central Hermite moments       (Sec. 2.1.3)
//   T f_eq = (rho, 0, ..., 0) with the full-expansion f_eq     (Eq. Hermite_coeff_eq)
//   Bouzidi interpolated bounce-back, q = |x_f - x_s| / |c|    (Sec. 2.1.4)
//
// GB300 design:
//   * Populations are SoA, pop[i][slot], slot = brick * 64 + local cell of a 4x4x4 brick; only
//     bricks with fluid are stored.  One thread per slot, one CTA per four bricks; the brick
//     neighbour table of the CTA is staged in shared memory, so streaming costs no per-cell
//     neighbour index (27 x 4 B per brick instead of per cell).
//   * Pull scheme with two arrays (A -> B): every thread reads its 27 incoming populations
//     (coalesced along x within a brick row) and writes its 27 outgoing ones to its own slot
//     (fully coalesced).
//   * A per-slot 32-bit word carries the wall mask and the cell kind, so bulk cells take no
//     boundary branch; wall cells read one aux index and their q values.
//   * Arithmetic is FP32 on deviations d_i = f_i - w_i throughout (moments, transforms,
//     relaxation, closures): the O(1) rest-state weights never enter a rounding, which keeps
//     FP32 results within 1e-5 of the FP64 oracle over thousands of steps.
//   * The 27x27 transform is applied as three passes of nine 1-D three-point transforms
//     (T = M(u_x) (x) M(u_y) (x) M(u_z)), forward and inverse, about 500 FP32 flops per cell.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr float CS2 = 1.0f / 3.0f;

// ------------------------------------------------------------------------------ storage
// FP32 stores d_i; FP16 / BF16 store d_i / w_i.
template <int ST>
struct Store;

template <>
struct Store<LBM_STORE_FP32> {
    using T = float;
    static __device__ __forceinline__ float load(const void* p, int64_t n, int i, int64_t s)
    {
        return __ldg(static_cast<const float*>(p) + (int64_t)i * n + s);
    }
    static __device__ __forceinline__ float load_at(const void* p, int, uint32_t off)
    {
        return __ldg(static_cast<const float*>(p) + off);
    }
    static __device__ __forceinline__ void store(void* p, int64_t n, int i, int64_t s, float v)
    {
        static_cast<float*>(p)[(int64_t)i * n + s] = v;
    }
};

template <>
struct Store<LBM_STORE_FP16> {
    using T = __half;
    static __device__ __forceinline__ float load(const void* p, int64_t n, int i, int64_t s)
    {
        const __half h = __ldg(static_cast<const __half*>(p) + (int64_t)i * n + s);
        return w_of(i) * __half2float(h);
    }
    static __device__ __forceinline__ float load_at(const void* p, int i, uint32_t off)
    {
        return w_of(i) * __half2float(__ldg(static_cast<const __half*>(p) + off));
    }
    static __device__ __forceinline__ void store(void* p, int64_t n, int i, int64_t s, float v)
    {
        static_cast<__half*>(p)[(int64_t)i * n + s] = __float2half_rn(v * inv_w_of(i));
    }
};

template <>
struct Store<LBM_STORE_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float load(const void* p, int64_t n, int i, int64_t s)
    {
        const __nv_bfloat16 h = __ldg(static_cast<const __nv_bfloat16*>(p) + (int64_t)i * n + s);
        return w_of(i) * __bfloat162float(h);
    }
    static __device__ __forceinline__ float load_at(const void* p, int i, uint32_t off)
    {
        return w_of(i) * __bfloat162float(__ldg(static_cast<const __nv_bfloat16*>(p) + off));
    }
    static __device__ __forceinline__ void store(void* p, int64_t n, int i, int64_t s, float v)
    {
        static_cast<__nv_bfloat16*>(p)[(int64_t)i * n + s] = __float2bfloat16_rn(v * inv_w_of(i));
    }
};

// ------------------------------------------------------------------------------ gather
// Open-boundary closure of an inlet (velocity) or outlet (density) cell on an axis-aligned face
// with inward normal n = sign e_axis, in deviation form.  Known: c.n <= 0.  With
// D = sum_{c.n=0} d + 2 sum_{c.n<0} d (and sum_{c.n=0} w + 2 sum_{c.n<0} w = 1):
//   inlet:  u.n = U phi, rho = (1 + D)/(1 - u.n);   outlet: rho = rho_out, u.n = 1 - (1 + D)/rho.
// Both are evaluated as deviations from 1 (rho - 1 = (D + u.n)/(1 - u.n), u.n = (rho_out - 1 - D)/rho_out).
// The nine unknowns (c.n = +1) by non-equilibrium bounce-back with the full equilibrium; since
// u has no tangential part, f_eq_i - f_eq_opp(i) = 6 w_i rho u.n.  Then the tangential momentum
// is zeroed by d_i += c_it D_t / 6, D_t = -sum_j c_jt d_j, which leaves mass and normal
// momentum unchanged.
__device__ __forceinline__ void close_open(float (&d)[Q], int kind, int axis, int sgn, float phi,
                                           float U, float rho_out, float drho_out)
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
        // u.n = 1 - (1 + D)/rho_out written as (drho_out - D)/rho_out, drho_out = rho_out - 1
        // from the host in FP64, so that D is never rounded against 1
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

// Pull the 27 populations of level n into `d` (deviations) for the fluid cell at `slot`:
// f_i(x, n) = f*_i(x - c_i, n - 1) from `src`, then the wall rules on masked links and the
// open-boundary closure.  `nbrow` is the 27-entry neighbour row of the cell's brick.
// Every lane issues all 27 loads unconditionally: on a wall link the address is redirected to
// the cell's own opposite population, which is halfway bounce-back, f_i(x) = f*_opp(i)(x).  The
// loads are independent, so they are all in flight together.
template <int ST>
__device__ __forceinline__ void gather(const DomainView& v, const void* __restrict__ src,
                                       const int32_t* nbrow, uint32_t slot, uint32_t word,
                                       const LevelArgs& a, float (&d)[Q])
{
    using S = Store<ST>;
    const uint32_t n = (uint32_t)v.n_slots;
    const int l = (int)(slot & (BRICK_CELLS - 1));
    const int lx = l & 3, ly = (l >> 2) & 3, lz = l >> 4;
    const uint32_t wm = word & WORD_WALL_MASK;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sx = lx - cx_of(i), sy = ly - cy_of(i), sz = lz - cz_of(i);
        // sx in [-1, 4]: the arithmetic shift gives the brick offset -1, 0 or +1
        const int ob = 13 + (sx >> 2) + 3 * (sy >> 2) + 9 * (sz >> 2);
        const uint32_t nb = (uint32_t)nbrow[ob];
        const uint32_t s = nb * BRICK_CELLS + (uint32_t)((sx & 3) + ((sy & 3) << 2) + ((sz & 3) << 4));
        const bool wall = (wm >> i) & 1u;
        const uint32_t off = wall ? (uint32_t)(Q - 1 - i) * n + slot : (uint32_t)i * n + s;
        d[i] = S::load_at(src, i, off);
    }
    if (wm == 0u) return;
    const int kind = (int)((word >> WORD_KIND_SHIFT) & 3u);
    if (kind == KIND_BOUZIDI) {
        // Sec. 2.1.4 in pull form with beta = opp(alpha) pointing into the wall:
        //   q <  1/2: f_a(x) = 2q f*_b(x) + (1 - 2q) f*_b(x + c_a)  [= the value pulled for b]
        //   q >= 1/2: f_a(x) = f*_b(x)/(2q) + (2q - 1)/(2q) f*_a(x)
        // with halfway bounce-back kept if x + c_a is not fluid in the first branch.
        const int64_t rec = v.aux[slot];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (!(wm & (1u << i))) continue;
            const float q = __ldg(v.bq + (int64_t)i * v.n_bq + rec);
            if (q > 0.0f) {
                if (q < 0.5f) {
                    if (!(wm & (1u << (Q - 1 - i)))) d[i] = 2.0f * q * d[i] + (1.0f - 2.0f * q) * d[Q - 1 - i];
                } else {
                    const float inv2q = 0.5f / q;
                    d[i] = inv2q * d[i] + (1.0f - inv2q) * S::load(src, v.n_slots, i, slot);
                }
            }
        }
    } else if (kind >= KIND_INLET) {
        const int64_t rec = v.aux[slot];
        close_open(d, kind, v.io_axis[rec], v.io_sign[rec], v.io_phi[rec], a.U, a.rho_out, a.drho_out);
    }
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

// ------------------------------------------------------------------------------ kernels
template <int ST, int BRICKS, int MINB>
__global__ void __launch_bounds__(BRICKS * BRICK_CELLS, MINB)
    k_step(DomainView v, const void* __restrict__ src, void* __restrict__ dst, LevelArgs a)
{
    __shared__ int32_t s_nbr[BRICKS * Q];
    const int64_t brick0 = (int64_t)blockIdx.x * BRICKS;
    for (int t = threadIdx.x; t < BRICKS * Q; t += blockDim.x)
        s_nbr[t] = (brick0 + t / Q < v.n_bricks) ? __ldg(v.nbr + brick0 * Q + t) : -1;
    __syncthreads();
    const uint32_t slot = (uint32_t)(brick0 * BRICK_CELLS) + threadIdx.x;
    if (slot >= (uint32_t)v.n_slots) return;
    const uint32_t word = __ldg(v.word + slot);
    if (!(word & WORD_FLUID)) return;
    float d[Q];
    gather<ST>(v, src, s_nbr + (threadIdx.x / BRICK_CELLS) * Q, slot, word, a, d);
    collide(d, a);
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<ST>::store(dst, v.n_slots, i, slot, d[i]);
}

template <int ST>
__global__ void __launch_bounds__(256)
    k_macroscopic(DomainView v, const void* __restrict__ src, LevelArgs a, const int32_t* fl_slot,
                  const int32_t* fl_box, int64_t n_fluid, int dense, float* rho, float* u, int64_t n_out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_fluid) return;
    const int64_t slot = fl_slot[k];
    const uint32_t word = v.word[slot];
    float d[Q];
    gather<ST>(v, src, v.nbr + (slot / BRICK_CELLS) * Q, (uint32_t)slot, word, a, d);
    const Moments M = moments(d, a.g);
    const int64_t o = dense ? (int64_t)fl_box[k] : k;
    rho[o] = M.rho;
    u[o] = M.ux;
    u[n_out + o] = M.uy;
    u[2 * n_out + o] = M.uz;
}

// Post-collision populations of level n - 1 := f_eq(rho, u) (full expansion, product form),
// written as deviations: d_i = rho (prod psi - w_i) + (rho - 1) w_i with
// prod psi - w = dpx psi_y psi_z + w1x dpy psi_z + w1x w1y dpz, dpsi(0) = -u^2,
// dpsi(+-1) = (+-u + u^2)/2.
template <int ST>
__global__ void __launch_bounds__(256)
    k_init_equilibrium(int64_t n_slots, void* dst, const int32_t* fl_slot, const int32_t* fl_box,
                       int64_t n_fluid, const float* rho_in, const float* u_in, int64_t n_box)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_fluid) return;
    const int64_t b = fl_box[k];
    const int64_t slot = fl_slot[k];
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
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ix = cx_of(i) + 1, iy = cy_of(i) + 1, iz = cz_of(i) + 1;
        const float w1x = w1_of(cx_of(i)), w1y = w1_of(cy_of(i));
        const float dprod = dp[0][ix] * ps[1][iy] * ps[2][iz] + w1x * dp[1][iy] * ps[2][iz] +
                            w1x * w1y * dp[2][iz];
        const float dv = fmaf(rho, dprod, (rho - 1.0f) * w_of(i));
        Store<ST>::store(dst, n_slots, i, slot, dv);
    }
}

// FP64 diagnostics: per-block partial sums in a fixed order, then one block reduces them in a
// fixed order (reproducible run to run).
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

template <int ST>
__global__ void __launch_bounds__(DIAG_THREADS)
    k_diagnostics(DomainView v, const void* __restrict__ src, LevelArgs a, const int32_t* fl_slot,
                  int64_t n_fluid, double* partials)
{
    __shared__ double sh[(DIAG_THREADS / 32) * DIAG_FIELDS];
    double x[DIAG_FIELDS] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t k = (int64_t)blockIdx.x * DIAG_THREADS + threadIdx.x;
    if (k < n_fluid) {
        const int64_t slot = fl_slot[k];
        const uint32_t word = v.word[slot];
        float d[Q];
        gather<ST>(v, src, v.nbr + (slot / BRICK_CELLS) * Q, (uint32_t)slot, word, a, d);
        const Moments M = moments(d, a.g);
        const bool finite = isfinite(M.rho) && isfinite(M.ux) && isfinite(M.uy) && isfinite(M.uz);
        if (finite) {
            x[0] = (double)M.rho;
            const int kind = (int)((word >> WORD_KIND_SHIFT) & 3u);
            if (kind >= KIND_INLET) {
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

__global__ void __launch_bounds__(DIAG_THREADS)
    k_diagnostics_final(const double* partials, int64_t n_blocks, lbm_diagnostics* out)
{
    __shared__ double sh[(DIAG_THREADS / 32) * DIAG_FIELDS];
    double x[DIAG_FIELDS] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t b = threadIdx.x; b < n_blocks; b += DIAG_THREADS)
        for (int f = 0; f < DIAG_FIELDS; ++f) {
            const double p = partials[b * DIAG_FIELDS + f];
            x[f] = (f == 3) ? fmax(x[f], p) : x[f] + p;
        }
    block_reduce5(x, sh);
    if (threadIdx.x == 0) {
        out->mass = x[0];
        out->flux_in = x[1];
        out->flux_out = x[2];
        out->max_u = x[3];
        out->n_nonfinite = (int64_t)x[4];
    }
}

int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

// ------------------------------------------------------------------------------ launchers
// Launch configurations of the step kernel: (bricks per CTA, minimum resident CTAs per SM).
// The second number sets the register budget: 65536 / (threads * CTAs).
namespace {
template <int ST, int BRICKS, int MINB>
cudaError_t launch_step_t(const DomainView& v, const void* src, void* dst, const LevelArgs& a, cudaStream_t stream)
{
    const int grid = grid_for(v.n_bricks, BRICKS);
    k_step<ST, BRICKS, MINB><<<grid, BRICKS * BRICK_CELLS, 0, stream>>>(v, src, dst, a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_step_cfg(int config, const DomainView& v, const void* src, void* dst, const LevelArgs& a,
                            cudaStream_t stream)
{
    switch (config) {
    case 0: return launch_step_t<ST, 4, 2>(v, src, dst, a, stream);
    case 1: return launch_step_t<ST, 4, 3>(v, src, dst, a, stream);
    case 2: return launch_step_t<ST, 4, 4>(v, src, dst, a, stream);
    case 3: return launch_step_t<ST, 2, 6>(v, src, dst, a, stream);
    case 4: return launch_step_t<ST, 2, 8>(v, src, dst, a, stream);
    default: return launch_step_t<ST, 8, 1>(v, src, dst, a, stream);
    }
}
}  // namespace

const char* launch_config_name(int config)
{
    static const char* names[N_LAUNCH_CONFIGS] = {"256x2", "256x3", "256x4", "128x6", "128x8", "512x1"};
    return (config >= 0 && config < N_LAUNCH_CONFIGS) ? names[config] : "?";
}

cudaError_t launch_step(int storage, int config, const DomainView& v, const void* src, void* dst,
                        const LevelArgs& a, cudaStream_t stream)
{
    if (v.n_bricks == 0) return cudaSuccess;
    switch (storage) {
    case LBM_STORE_FP32: return launch_step_cfg<LBM_STORE_FP32>(config, v, src, dst, a, stream);
    case LBM_STORE_FP16: return launch_step_cfg<LBM_STORE_FP16>(config, v, src, dst, a, stream);
    default: return launch_step_cfg<LBM_STORE_BF16>(config, v, src, dst, a, stream);
    }
}

cudaError_t launch_macroscopic(int storage, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, const int32_t* fl_box, int64_t n_fluid, int dense,
                               float* rho, float* u, int64_t n_out, cudaStream_t stream)
{
    if (n_fluid == 0) return cudaSuccess;
    const int grid = grid_for(n_fluid, 256);
    switch (storage) {
    case LBM_STORE_FP32:
        k_macroscopic<LBM_STORE_FP32><<<grid, 256, 0, stream>>>(v, src, a, fl_slot, fl_box, n_fluid, dense, rho, u, n_out);
        break;
    case LBM_STORE_FP16:
        k_macroscopic<LBM_STORE_FP16><<<grid, 256, 0, stream>>>(v, src, a, fl_slot, fl_box, n_fluid, dense, rho, u, n_out);
        break;
    default:
        k_macroscopic<LBM_STORE_BF16><<<grid, 256, 0, stream>>>(v, src, a, fl_slot, fl_box, n_fluid, dense, rho, u, n_out);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(int storage, int64_t n_slots, void* dst, const int32_t* fl_slot,
                                    const int32_t* fl_box, int64_t n_fluid, const float* rho, const float* u,
                                    int64_t n_box, cudaStream_t stream)
{
    if (n_fluid == 0) return cudaSuccess;
    const int grid = grid_for(n_fluid, 256);
    switch (storage) {
    case LBM_STORE_FP32:
        k_init_equilibrium<LBM_STORE_FP32><<<grid, 256, 0, stream>>>(n_slots, dst, fl_slot, fl_box, n_fluid, rho, u, n_box);
        break;
    case LBM_STORE_FP16:
        k_init_equilibrium<LBM_STORE_FP16><<<grid, 256, 0, stream>>>(n_slots, dst, fl_slot, fl_box, n_fluid, rho, u, n_box);
        break;
    default:
        k_init_equilibrium<LBM_STORE_BF16><<<grid, 256, 0, stream>>>(n_slots, dst, fl_slot, fl_box, n_fluid, rho, u, n_box);
        break;
    }
    return cudaGetLastError();
}

int64_t diagnostics_blocks(int64_t n_fluid) { return n_fluid == 0 ? 1 : (n_fluid + DIAG_THREADS - 1) / DIAG_THREADS; }

cudaError_t launch_diagnostics(int storage, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, int64_t n_fluid, double* partials, lbm_diagnostics* out,
                               cudaStream_t stream)
{
    const int64_t nb = diagnostics_blocks(n_fluid);
    switch (storage) {
    case LBM_STORE_FP32:
        k_diagnostics<LBM_STORE_FP32><<<(int)nb, DIAG_THREADS, 0, stream>>>(v, src, a, fl_slot, n_fluid, partials);
        break;
    case LBM_STORE_FP16:
        k_diagnostics<LBM_STORE_FP16><<<(int)nb, DIAG_THREADS, 0, stream>>>(v, src, a, fl_slot, n_fluid, partials);
        break;
    default:
        k_diagnostics<LBM_STORE_BF16><<<(int)nb, DIAG_THREADS, 0, stream>>>(v, src, a, fl_slot, n_fluid, partials);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diagnostics_final<<<1, DIAG_THREADS, 0, stream>>>(partials, nb, out);
    return cudaGetLastError();
}

}  // namespace lbm
