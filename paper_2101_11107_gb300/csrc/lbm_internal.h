// lbm_internal.h -- shared declarations of the CUDA library (device views, launch arguments,
// stencil constants).  Not part of the public C-ABI (include/lbm.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

// An NVTX range over a scope: entry points that enqueue or run device work mark themselves on
// the host timeline of a profiler (nvtx3 is header-only; without a tool attached a push/pop is
// a test of a null function pointer).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// D3Q27, i = (cx+1) + 3 (cy+1) + 9 (cz+1); opposite = 26 - i.  Weights are the products of the
// D1Q3 weights (2/3, 1/6, 1/6): 8/27, 2/27, 1/54, 1/216 by |c|^2.
constexpr int Q = 27;
__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }
__host__ __device__ constexpr float w1_of(int c) { return c == 0 ? 2.0f / 3.0f : 1.0f / 6.0f; }
__host__ __device__ constexpr float w_of(int i)
{
    return w1_of(cx_of(i)) * w1_of(cy_of(i)) * w1_of(cz_of(i));
}
__host__ __device__ constexpr float inv_w_of(int i) { return 1.0f / w_of(i); }
// number of nonzero components of c_i, and 2^-k
__host__ __device__ constexpr int nnz_of(int i) { return (cx_of(i) != 0) + (cy_of(i) != 0) + (cz_of(i) != 0); }
__host__ __device__ constexpr float pow2_neg(int k) { return k == 0 ? 1.0f : k == 1 ? 0.5f : k == 2 ? 0.25f : 0.125f; }
// corner of the positive part p_i = max(c_i, 0), and of p_opp(i) = max(-c_i, 0): e = px + 2py + 4pz
__host__ __device__ constexpr int corner_pos(int i) { return (cx_of(i) > 0) + 2 * (cy_of(i) > 0) + 4 * (cz_of(i) > 0); }
__host__ __device__ constexpr int corner_neg(int i) { return (cx_of(i) < 0) + 2 * (cy_of(i) < 0) + 4 * (cz_of(i) < 0); }

// Geometry is stored in bricks of BX x BY x BZ = 64 cells (powers of two; 4 x 4 x 4 unless the
// library is built with LBM_BRICK_X/Y/Z); a population slot is brick * 64 + lx + BX (ly + BY lz).
// Bricks holding fluid ("active", updated every step) come first; the esoteric-twist layout adds
// the bricks at offsets {0,1}^3 of active bricks ("halo", storage only).  A warp covers half a
// brick (lz < BZ / 2 or lz >= BZ / 2).
#ifndef LBM_BRICK_X
#define LBM_BRICK_X 4
#define LBM_BRICK_Y 4
#define LBM_BRICK_Z 4
#endif
constexpr int BX = LBM_BRICK_X, BY = LBM_BRICK_Y, BZ = LBM_BRICK_Z;
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }
constexpr int LBX = ilog2(BX), LBY = ilog2(BY), LBZ = ilog2(BZ);
constexpr int BRICK_CELLS = 64;
static_assert(BX * BY * BZ == BRICK_CELLS && (1 << LBX) == BX && (1 << LBY) == BY && (1 << LBZ) == BZ && BZ >= 2,
              "a brick is 64 cells, each extent a power of two, at least two layers along z");
constexpr int BRICK_EXT[3] = {BX, BY, BZ};
// local index of (lx, ly, lz) in a brick; (lx, ly, lz) of a local index
__host__ __device__ constexpr int brick_local(int lx, int ly, int lz) { return lx | (ly << LBX) | (lz << (LBX + LBY)); }

// Per-slot cell word (active bricks).
//   bits 0..26  wall mask: bit i set <=> the pull source x - c_i is not a fluid cell
//   bits 27..28 kind (plain / Bouzidi / inlet / outlet)
//   bit 29      the cell relaxes with its own second-order rate s2_cell[slot]
//   bit 31      the slot is a fluid cell (updated every step); solid slots have word 0
constexpr uint32_t WORD_FLUID = 1u << 31;
constexpr uint32_t WORD_OWN_TAU = 1u << 29;  // the cell has its own relaxation time (s2_cell)
constexpr uint32_t WORD_WALL_MASK = (1u << 27) - 1u;
constexpr int WORD_KIND_SHIFT = 27;
enum CellKind { KIND_PLAIN = 0, KIND_BOUZIDI = 1, KIND_INLET = 2, KIND_OUTLET = 3 };

// Geometry of a domain on the device.
struct DomainView {
    int64_t n_slots;        // population stride: 64 * (active + halo bricks)
    int64_t n_bricks;       // active bricks
    const int32_t* nbr;     // A-B:  [n_bricks][27] brick at offset (ox,oy,oz) in {-1,0,1}^3, -1 none
    const int32_t* nb8;     // twist: [n_bricks][8] brick at offset (ex,ey,ez) in {0,1}^3, never -1
    const uint32_t* word;   // [64 n_bricks]
    const int32_t* aux;     // [64 n_bricks] record of a Bouzidi or open-boundary cell
    const float* s2_cell;   // [64 n_bricks] second-order rate of cells with WORD_OWN_TAU
    const float* bq;        // [n_bq] q of every wall link of the Bouzidi cells, packed per cell: cell
                            // (aux record a, wall mask wm) owns a .. a + popc(wm) - 1 in direction
                            // order (0: halfway bounce-back on that link)
    void* side;             // twist: [n_bq] f*_i of the previous step, same packing (storage type)
    int64_t n_bq;           // packed links (at least 1)
    const float* io_phi;    // [n_io] inflow profile factor 2 (1 - r^2/R^2)
    const int8_t* io_axis;  // [n_io] inward normal axis
    const int8_t* io_sign;  // [n_io] inward normal sign
    int64_t n_io;
};

// FP64 running sums of (rho, ux, uy, uz) of one fluid cell.
struct alignas(32) Sum4 {
    double x, y, z, w;
};

// Per-launch arguments of a time level n.
struct LevelArgs {
    float g[3];    // body acceleration g(n)
    float U;       // inflow U(n) for the open-boundary closure of level n
    float s2, s3, s4, s5, s6;  // relaxation rates by moment order
    float rho_out;
    float drho_out;  // rho_out - 1, rounded once from FP64
    int parity;      // n & 1 (esoteric twist)
    int coll;        // collision kernel: COLL_CHM, COLL_CHM_FAST (every 3rd..6th-order rate is
                     // 1: the step kernel skips those moments), COLL_SRT2, COLL_TRT2
    float wm;        // SRT2 / TRT2: rate of the odd parts (SRT2: = s2)
    float magic;     // TRT2: Lambda, for cells with their own tau
};

// Barrier state of a persistent batched launch (cleared before each launch).
struct GridBarrier {
    unsigned int count;  // arrivals so far in this launch (step s completes at (s + 1) * gridDim.x)
    unsigned int fail;   // 1: a wait gave up; the populations are no longer a valid state
};

// One domain of a batched launch.
struct BatchEntry {
    DomainView view;
    void* pop;  // the domain's in-place population array
};

constexpr int N_LAUNCH_CONFIGS = 8;

// collision kernels (the `coll` of LevelArgs and the COLL template parameter of the step kernels)
constexpr int COLL_CHM = 0, COLL_CHM_FAST = 1, COLL_SRT2 = 2, COLL_TRT2 = 3;
constexpr int DEFAULT_LAUNCH_CONFIG = 2;  // 128 threads, 6 CTAs per SM

// Launchers, one set per storage precision (lbm_step_<storage>.cu).  All enqueue on `stream`
// and return the launch status.
struct Launchers {
    cudaError_t (*step)(int scheme, int config, const DomainView& v, const void* src, void* dst,
                        const LevelArgs& a, cudaStream_t stream);
    cudaError_t (*macroscopic)(int scheme, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, const int32_t* fl_box, int64_t n_fluid, int dense,
                               float* rho, float* u, int64_t n_out, cudaStream_t stream);
    cudaError_t (*init_equilibrium)(int scheme, const DomainView& v, void* dst, int parity_prev,
                                    const int32_t* fl_slot, const int32_t* fl_box, int64_t n_fluid,
                                    const float* rho, const float* u, int64_t n_box, cudaStream_t stream);
    cudaError_t (*diagnostics)(int scheme, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, int64_t n_fluid, double* partials, cudaStream_t stream);
    // twist only: every domain of the batch one step; args[d] are domain d's level arguments;
    // parity: the parity every args[d].parity has (0 or 1), or -1 if they differ
    cudaError_t (*step_batch)(int config, const BatchEntry* ent, const int64_t* brick_start, int n_dom,
                              int64_t total_bricks, const LevelArgs* args, int coll, int parity,
                              cudaStream_t stream);
    // learned-corrector velocity shift of the post-collision populations of the previous level
    cudaError_t (*apply_du)(int scheme, const DomainView& v, void* pop, int parity_prev, const int32_t* fl_slot,
                            const int32_t* fl_box, int64_t n_fluid, const float* rho, const float* u, const float* du,
                            int64_t n_box, cudaStream_t stream);
    // running-mean accumulation (FP64 sums of rho, u per fluid cell) and point probes
    cudaError_t (*mean_sample)(int scheme, const DomainView& v, const void* src, const LevelArgs& a,
                               const int32_t* fl_slot, int64_t n_fluid, Sum4* sums, cudaStream_t stream);
    cudaError_t (*probe)(int scheme, const DomainView& v, const void* src, const LevelArgs& a, const int32_t* fl_slot,
                         int64_t n_fluid, const int64_t* idx, int n, float4* out, cudaStream_t stream);
    // bounds-checked build (LBM_DEBUG): code of the first out-of-range access the kernels of this
    // storage precision skipped since the last call (0: none; always 0 in the default build)
    unsigned (*debug_fault)();
    // persistent batched step: `steps` steps of every domain in one cooperative launch, a grid
    // barrier (waits bounded by limit_ns) between steps; args[s][d]; parity0: the parity every
    // domain has at step 0, or -1
    cudaError_t (*step_batch_persistent)(const BatchEntry* ent, const int64_t* brick_start, int n_dom,
                                         int64_t total_bricks, const LevelArgs* args, int coll, int parity0, int steps,
                                         GridBarrier* bar, uint64_t limit_ns, cudaStream_t stream);
};
// storage-independent output of the running means (lbm_metrics.cu)
cudaError_t launch_mean_out(const Sum4* sums, const int32_t* fl_box, int64_t n_fluid, int64_t n_samples, int dense,
                            float* rho, float* u, int64_t n_out, cudaStream_t stream);
const Launchers& launchers_fp32();
const Launchers& launchers_fp16();
const Launchers& launchers_bf16();
const Launchers& launchers(int storage);

// halo exchange of a slab decomposition: the 9 directions crossing a face, in increasing i
struct HaloDirs {
    int8_t d[9];
};
// pack: buf[j][p] = pop[dirs[j]][slot[p]] (0 where slot[p] < 0); unpack: the reverse where
// slot[p] >= 0; values of bytes_per_value bytes, copied bit for bit
cudaError_t launch_halo_copy(int bytes_per_value, bool pack, void* pop, int64_t n_slots, const int32_t* slot,
                             int64_t area, const HaloDirs& dirs, void* buf, cudaStream_t stream);

int64_t diagnostics_blocks(int64_t n_fluid);
cudaError_t launch_diagnostics_final(const double* partials, int64_t n_blocks, lbm_diagnostics* out,
                                     cudaStream_t stream);
const char* launch_config_name(int config);

// Read access to a domain's device state for entry points defined outside lbm_domain.cu.
struct DomainAccess {
    int storage, scheme;
    const DomainView* view;
    const void* src;      // populations of the current level
    LevelArgs args;       // arguments of the current level
    const int32_t* fl_slot;
    int64_t n_fluid;
    int64_t time;
    cudaStream_t stream;
    uint64_t serial;  // unique per domain of the process
};
bool domain_access(const lbm_domain* dom, DomainAccess* out);
// the dense export of lbm_get_macroscopic on the domain's stream; clear = false leaves the
// cells that are not fluid as they are (a caller whose arrays already hold this domain's zeros
// there)
cudaError_t enqueue_macroscopic_dense(lbm_domain* dom, float* rho, float* u, bool clear);
// the velocity correction of lbm_apply_velocity_correction with the current level's rho and u
// already exported (dense device arrays, as lbm_get_macroscopic writes them): enqueued on the
// domain's stream
cudaError_t enqueue_velocity_correction(lbm_domain* dom, const float* rho, const float* u, const float* du);
// sets the calling thread's lbm_last_error() message
void set_last_error(const char* msg);

}  // namespace lbm
