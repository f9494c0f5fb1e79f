// lbm_domain.cu -- host side of the C-ABI (include/lbm.h): validation, the brick layout of a
// voxel domain, device memory through the caller's allocator, time levels, checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

lbm_status fail(lbm_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

lbm_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// LBM_DEBUG builds: STATE if a kernel skipped an out-of-range access (after the stream has
// been synchronised); the default build returns OK without a device call
lbm_status debug_status(int storage)
{
#ifdef LBM_DEBUG
    const unsigned code = launchers(storage).debug_fault();
    if (code)
        return fail(LBM_ERR_STATE, "LBM_DEBUG: a kernel skipped an out-of-range access (check " + std::to_string(code) + ")");
#else
    (void)storage;
#endif
    return LBM_OK;
}

}  // namespace

struct lbm_domain {
    int32_t nx = 0, ny = 0, nz = 0;
    uint64_t serial = 0;  // unique per domain of the process (never reused, unlike an address)
    lbm_params params{};
    int64_t n_fluid = 0, n_bricks = 0, n_store_bricks = 0, n_slots = 0, n_bq = 0, n_io = 0, n_wall = 0;
    int64_t n_blinks = 0;  // wall links of the Bouzidi cells (length of the packed link lists)
    DomainView view{};
    int32_t* d_fl_slot = nullptr;
    int32_t* d_fl_box = nullptr;
    void* d_pop[2] = {nullptr, nullptr};
    // A-B: d_pop[cur] holds the post-collision populations of level time - 1; esoteric twist:
    // d_pop[0] holds them in place, arranged for a read of parity time & 1
    int cur = 0;
    void* d_side = nullptr;  // twist: f* of q >= 1/2 Bouzidi links, one entry per packed link
    int launch_config = DEFAULT_LAUNCH_CONFIG;
    double* d_partials = nullptr;
    lbm_diagnostics* d_diag = nullptr;
    Sum4* d_mean = nullptr;  // running-mean sums (rho, ux, uy, uz) per fluid cell, FP64
    int64_t n_mean = 0;
    int64_t time = 0;
    // inflow waveform, tabulated over one period in FP64 and rounded to FP32
    bool has_wave = false;
    std::vector<float> wave;
    std::vector<double> wave_a, wave_b;
    double wave_period = 0.0, wave_peak = 0.0;
    cudaStream_t stream = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void* alloc_ctx = nullptr;
    std::vector<void*> owned;
    int64_t device_bytes = 0;
    float* d_corr_stage = nullptr;  // rho, u and a staged du for the velocity correction (lazy)
    // halo layers (mask value 4, A-B only): per box face, the slots of the halo cells and of the
    // fluid cells one layer inside, at every position of the face (-1: none)
    int64_t n_halo = 0;
    int32_t* d_halo_slot[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int32_t* d_inner_slot[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t face_area[6] = {0, 0, 0, 0, 0, 0};
    // host copies kept for checkpoints
    uint64_t geometry_hash = 0;

    int bytes_per_value() const { return params.storage == LBM_STORE_FP32 ? 4 : 2; }
    size_t pop_bytes() const { return (size_t)Q * (size_t)n_slots * (size_t)bytes_per_value(); }
    size_t side_bytes() const { return (size_t)std::max<int64_t>(n_blinks, 1) * (size_t)bytes_per_value(); }
    bool twist() const { return params.scheme == LBM_SCHEME_ESOTERIC; }
    void* src() const { return d_pop[twist() ? 0 : cur]; }
    void* dst() const { return d_pop[twist() ? 0 : 1 - cur]; }

    void* dev_alloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        void* p = nullptr;
        if (alloc) {
            p = alloc(bytes, alloc_ctx);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) {
            owned.push_back(p);
            device_bytes += (int64_t)bytes;
        }
        return p;
    }

    // gives back one buffer obtained from dev_alloc
    void dev_free(void* p, size_t bytes)
    {
        auto it = std::find(owned.begin(), owned.end(), p);
        if (it == owned.end()) return;
        owned.erase(it);
        if (bytes) device_bytes -= (int64_t)((bytes + 255) & ~(size_t)255);
        if (release) release(p, alloc_ctx);
        else if (!alloc) cudaFree(p);
    }

    void release_all()
    {
        for (void* p : owned) {
            if (release) release(p, alloc_ctx);
            else if (!alloc) cudaFree(p);
        }
        owned.clear();
    }

    LevelArgs level_args(int64_t n) const
    {
        LevelArgs a{};
        for (int d = 0; d < 3; ++d)
            a.g[d] = (float)(params.force[d] + params.force_amp[d] * std::cos(params.force_omega * (double)n));
        a.U = 0.0f;
        if (has_wave && !wave.empty()) a.U = wave[(size_t)(n % (int64_t)wave.size())];
        a.s2 = (float)(1.0 / params.tau);
        a.s3 = (float)params.omega_hi[0];
        a.s4 = (float)params.omega_hi[1];
        a.s5 = (float)params.omega_hi[2];
        a.s6 = (float)params.omega_hi[3];
        a.rho_out = (float)params.rho_out;
        a.drho_out = (float)(params.rho_out - 1.0);
        a.parity = (int)(n & 1);
        const bool fast = params.omega_hi[0] == 1.0 && params.omega_hi[1] == 1.0 && params.omega_hi[2] == 1.0 &&
                          params.omega_hi[3] == 1.0;
        a.coll = params.collision == LBM_COLLISION_SRT2   ? COLL_SRT2
                 : params.collision == LBM_COLLISION_TRT2 ? COLL_TRT2
                 : fast                                   ? COLL_CHM_FAST
                                                          : COLL_CHM;
        a.magic = (float)params.trt_magic;
        a.wm = params.collision == LBM_COLLISION_TRT2
                   ? (float)(1.0 / (params.trt_magic / (params.tau - 0.5) + 0.5))
                   : a.s2;
        return a;
    }
};

namespace {

template <class T>
lbm_status upload(lbm_domain* D, T** dst, const std::vector<T>& src, const char* what)
{
    *dst = static_cast<T*>(D->dev_alloc(sizeof(T) * std::max<size_t>(src.size(), 1)));
    if (!*dst) return fail(LBM_ERR_OOM, std::string("allocation failed: ") + what);
    if (!src.empty()) {
        cudaError_t e = cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, D->stream);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    return LBM_OK;
}

uint64_t fnv1a(uint64_t h, const void* data, size_t n)
{
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

lbm_status check_params(const lbm_params& p)
{
    if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return fail(LBM_ERR_INVALID_ARG, "tau must be > 1/2");
    for (int k = 0; k < 4; ++k)
        if (!(p.omega_hi[k] > 0.0 && p.omega_hi[k] < 2.0))
            return fail(LBM_ERR_INVALID_ARG, "omega_hi must lie in (0, 2)");
    if (!(p.rho_out > 0.0) || !std::isfinite(p.rho_out)) return fail(LBM_ERR_INVALID_ARG, "rho_out must be > 0");
    if (p.storage < LBM_STORE_FP32 || p.storage > LBM_STORE_BF16) return fail(LBM_ERR_INVALID_ARG, "bad storage");
    if (p.scheme != LBM_SCHEME_AB && p.scheme != LBM_SCHEME_ESOTERIC) return fail(LBM_ERR_INVALID_ARG, "bad scheme");
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p.force[d]) || !std::isfinite(p.force_amp[d]))
            return fail(LBM_ERR_INVALID_ARG, "non-finite force");
    if (!std::isfinite(p.force_omega)) return fail(LBM_ERR_INVALID_ARG, "non-finite force_omega");
    if (p.collision < LBM_COLLISION_CHM_MRT || p.collision > LBM_COLLISION_TRT2)
        return fail(LBM_ERR_INVALID_ARG, "bad collision model");
    if (p.collision == LBM_COLLISION_TRT2 && !(p.trt_magic > 0.0 && std::isfinite(p.trt_magic)))
        return fail(LBM_ERR_INVALID_ARG, "trt_magic must be > 0");
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_params(lbm_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tau = 0.6;
    for (int k = 0; k < 4; ++k) p->omega_hi[k] = 1.0;
    p->rho_out = 1.0;
    p->storage = LBM_STORE_FP32;
    p->scheme = LBM_SCHEME_ESOTERIC;
    p->collision = LBM_COLLISION_CHM_MRT;
    p->trt_magic = 3.0 / 16.0;
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

lbm_status lbm_create_domain(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz, const int64_t* link_cell,
                             const uint8_t* link_dir, const double* link_q, int64_t n_links,
                             const double* inlet_center, double inlet_radius, const double* tau_cell,
                             const lbm_params* params, lbm_alloc_fn alloc, lbm_free_fn release, void* alloc_ctx,
                             void* cuda_stream, lbm_domain** out)
{
    g_last_error.clear();
    if (!out) return fail(LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!mask) return fail(LBM_ERR_INVALID_ARG, "mask is NULL");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(LBM_ERR_INVALID_ARG, "box extents must be positive");
    const int64_t n_box = (int64_t)nx * ny * nz;
    if (n_box >= ((int64_t)1 << 31)) return fail(LBM_ERR_INVALID_ARG, "box has 2^31 cells or more");
    if ((alloc == nullptr) != (release == nullptr))
        return fail(LBM_ERR_INVALID_ARG, "give both allocator callbacks or neither");
    if (n_links < 0 || (n_links > 0 && (!link_cell || !link_dir || !link_q)))
        return fail(LBM_ERR_INVALID_ARG, "bad link arrays");
    lbm_params P;
    if (params) P = *params;
    else lbm_default_params(&P);
    if (lbm_status s = check_params(P)) return s;
    const int n3[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        P.periodic[d] = P.periodic[d] ? 1 : 0;
        if (P.periodic[d] && n3[d] % BRICK_EXT[d] != 0)
            return fail(LBM_ERR_INVALID_ARG, "a periodic axis must have an extent that is a multiple of the brick's ("
                                                 + std::to_string(BRICK_EXT[d]) + ")");
    }

    // ---------------------------------------------------------------- bricks
    const int nbx = (nx + BX - 1) / BX, nby = (ny + BY - 1) / BY, nbz = (nz + BZ - 1) / BZ;
    const int64_t n_brick_box = (int64_t)nbx * nby * nbz;
    std::vector<int32_t> brick_id((size_t)n_brick_box, -1);
    int64_t n_fluid = 0, n_halo = 0;
    for (int64_t b = 0; b < n_box; ++b) {
        if (mask[b] > 4) return fail(LBM_ERR_INVALID_ARG, "mask value > 4");
        if (mask[b] == 4) ++n_halo;
        else if (mask[b]) ++n_fluid;
    }
    // halo cells: stored, filled by lbm_halo_unpack, never updated; A-B only, on a box face
    if (n_halo) {
        if (P.scheme != LBM_SCHEME_AB) return fail(LBM_ERR_INVALID_ARG, "halo cells (mask 4) need the A-B scheme");
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    if (mask[x + (int64_t)nx * (y + (int64_t)ny * z)] != 4) continue;
                    const int p[3] = {x, y, z};
                    bool on_face = false;
                    for (int d = 0; d < 3; ++d)
                        if (!P.periodic[d] && (p[d] == 0 || p[d] == n3[d] - 1)) on_face = true;
                    if (!on_face) return fail(LBM_ERR_INVALID_ARG, "a halo cell (mask 4) must lie on a non-periodic face");
                }
    }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                if (mask[x + (int64_t)nx * (y + (int64_t)ny * z)])
                    brick_id[(x >> LBX) + (int64_t)nbx * ((y >> LBY) + (int64_t)nby * (z >> LBZ))] = 0;
    // active bricks (holding fluid) are numbered first, in box order; then, for the esoteric
    // twist, every brick at an offset in {0,1}^3 of an active one (storage for the links of the
    // update's 8-cell corner), on a brick grid extended by one along non-periodic axes
    const int nb3[3] = {nbx, nby, nbz};
    int eb3[3];
    for (int d = 0; d < 3; ++d) eb3[d] = nb3[d] + (P.periodic[d] ? 0 : 1);
    const int64_t n_ext = (int64_t)eb3[0] * eb3[1] * eb3[2];
    std::vector<int32_t> store_id((size_t)n_ext, -1);
    auto ext_index = [&](int bx, int by, int bz) -> int64_t { return bx + (int64_t)eb3[0] * (by + (int64_t)eb3[1] * bz); };
    int64_t n_bricks = 0;
    std::vector<int32_t> brick_pos;  // (bx, by, bz) per active brick
    for (int64_t bb = 0; bb < n_brick_box; ++bb)
        if (brick_id[bb] == 0) {
            const int bx = (int)(bb % nbx), by = (int)((bb / nbx) % nby), bz = (int)(bb / ((int64_t)nbx * nby));
            brick_id[bb] = (int32_t)n_bricks;
            store_id[(size_t)ext_index(bx, by, bz)] = (int32_t)n_bricks++;
            brick_pos.push_back(bx);
            brick_pos.push_back(by);
            brick_pos.push_back(bz);
        }
    // brick at offset o of brick b along each axis, wrapped on periodic axes; -1 off the grid
    auto offset_brick = [&](int64_t b, int ox, int oy, int oz, bool extended) -> int64_t {
        int p[3] = {brick_pos[3 * b] + ox, brick_pos[3 * b + 1] + oy, brick_pos[3 * b + 2] + oz};
        for (int d = 0; d < 3; ++d) {
            const int lim = extended ? eb3[d] : nb3[d];
            if (p[d] < 0 || p[d] >= lim) {
                if (!P.periodic[d]) return -1;
                p[d] = (p[d] + nb3[d]) % nb3[d];
            }
        }
        return ext_index(p[0], p[1], p[2]);
    };
    int64_t n_store = n_bricks;
    const bool twist = P.scheme == LBM_SCHEME_ESOTERIC;
    std::vector<int32_t> nb8;
    if (twist) {
        nb8.assign((size_t)n_bricks * 8, -1);
        for (int64_t b = 0; b < n_bricks; ++b)
            for (int e = 0; e < 8; ++e) {
                const int64_t x = offset_brick(b, e & 1, (e >> 1) & 1, e >> 2, true);
                if (store_id[(size_t)x] < 0) store_id[(size_t)x] = (int32_t)n_store++;
                nb8[(size_t)b * 8 + e] = store_id[(size_t)x];
            }
    }
    const int64_t n_slots = n_store * BRICK_CELLS;
    // kernels address populations with 32-bit element offsets i * n_slots + slot
    if (n_slots * Q >= ((int64_t)1 << 32)) return fail(LBM_ERR_INVALID_ARG, "domain too large (27 x slots >= 2^32)");
    std::vector<int32_t> nbr;
    if (!twist) {
        nbr.assign((size_t)n_bricks * Q, -1);
        for (int64_t b = 0; b < n_bricks; ++b)
            for (int o = 0; o < Q; ++o) {
                const int64_t x = offset_brick(b, cx_of(o), cy_of(o), cz_of(o), false);
                if (x >= 0) nbr[(size_t)b * Q + o] = store_id[(size_t)x];
            }
    }
    auto slot_of = [&](int x, int y, int z) -> int64_t {
        const int64_t b = brick_id[(x >> LBX) + (int64_t)nbx * ((y >> LBY) + (int64_t)nby * (z >> LBZ))];
        return b * BRICK_CELLS + brick_local(x & (BX - 1), y & (BY - 1), z & (BZ - 1));
    };
    // fluid index of the box cell shifted by s * c_i, or -1 (solid / outside a non-periodic face)
    auto shifted_fluid = [&](int x, int y, int z, int i, int s) -> int64_t {
        int p[3] = {x + s * cx_of(i), y + s * cy_of(i), z + s * cz_of(i)};
        for (int d = 0; d < 3; ++d) {
            if (p[d] < 0 || p[d] >= n3[d]) {
                if (!P.periodic[d]) return -1;
                p[d] = (p[d] + n3[d]) % n3[d];
            }
        }
        const int64_t bi = p[0] + (int64_t)nx * (p[1] + (int64_t)ny * p[2]);
        return mask[bi] ? bi : -1;
    };

    // ---------------------------------------------------------------- cell words
    const int64_t n_active_slots = n_bricks * BRICK_CELLS;
    std::vector<uint32_t> word((size_t)n_active_slots, 0u);
    std::vector<int32_t> aux((size_t)n_active_slots, -1);
    std::vector<int32_t> fl_slot, fl_box;
    fl_slot.reserve((size_t)n_fluid);
    fl_box.reserve((size_t)n_fluid);
    int64_t n_wall = 0;
    std::vector<float> s2_cell(tau_cell ? (size_t)n_active_slots : 1, 0.0f);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t bi = x + (int64_t)nx * (y + (int64_t)ny * z);
                if (!mask[bi] || mask[bi] == 4) continue;  // halo cells: word 0 (stored, not updated)
                uint32_t w = WORD_FLUID;
                if (tau_cell && tau_cell[bi] != P.tau) {
                    if (!(tau_cell[bi] > 0.5) || !std::isfinite(tau_cell[bi]))
                        return fail(LBM_ERR_INVALID_ARG, "tau_cell must be > 1/2 at fluid cells");
                    w |= WORD_OWN_TAU;
                    s2_cell[(size_t)slot_of(x, y, z)] = (float)(1.0 / tau_cell[bi]);
                }
                for (int i = 0; i < Q; ++i)
                    if (i != 13 && shifted_fluid(x, y, z, i, -1) < 0) w |= 1u << i;
                if (w & WORD_WALL_MASK) ++n_wall;
                const int64_t s = slot_of(x, y, z);
                word[(size_t)s] = w;
                fl_slot.push_back((int32_t)s);
                fl_box.push_back((int32_t)bi);
            }

    // ---------------------------------------------------------------- open boundaries
    std::vector<float> io_phi;
    std::vector<int8_t> io_axis, io_sign;
    std::vector<std::pair<int64_t, int64_t>> io_cells;  // (slot, box index), sorted by slot
    for (int64_t k = 0; k < n_fluid; ++k)
        if (mask[fl_box[(size_t)k]] >= 2) io_cells.push_back({fl_slot[(size_t)k], fl_box[(size_t)k]});
    std::sort(io_cells.begin(), io_cells.end());
    for (const auto& c : io_cells) {
        const int64_t bi = c.second;
        const int p[3] = {(int)(bi % nx), (int)((bi / nx) % ny), (int)(bi / ((int64_t)nx * ny))};
        int faces = 0, ax = -1, sg = 0;
        for (int d = 0; d < 3; ++d) {
            if (P.periodic[d]) continue;
            if (p[d] == 0) { ++faces; ax = d; sg = +1; }
            if (p[d] == n3[d] - 1) { ++faces; ax = d; sg = -1; }
        }
        if (faces != 1) return fail(LBM_ERR_INVALID_ARG, "inlet/outlet cell not on exactly one non-periodic face");
        float phi = 0.0f;
        if (mask[bi] == 2) {
            if (!inlet_center || !(inlet_radius > 0.0))
                return fail(LBM_ERR_INVALID_ARG, "inlet cells need inlet_center and inlet_radius > 0");
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                if (d == ax) continue;
                const double dx = p[d] + 0.5 - inlet_center[d];
                r2 += dx * dx;
            }
            const double v = 2.0 * (1.0 - r2 / (inlet_radius * inlet_radius));
            phi = (float)(v > 0.0 ? v : 0.0);
        }
        const int32_t rec = (int32_t)io_phi.size();
        io_phi.push_back(phi);
        io_axis.push_back((int8_t)ax);
        io_sign.push_back((int8_t)sg);
        word[(size_t)c.first] |= (uint32_t)(mask[bi] == 2 ? KIND_INLET : KIND_OUTLET) << WORD_KIND_SHIFT;
        aux[(size_t)c.first] = rec;
    }

    // ---------------------------------------------------------------- Bouzidi links
    std::vector<std::pair<int64_t, std::pair<int, float>>> lk;  // (slot, (alpha, q))
    lk.reserve((size_t)n_links);
    for (int64_t l = 0; l < n_links; ++l) {
        const int64_t bi = link_cell[l];
        const int beta = link_dir[l];
        const double q = link_q[l];
        if (bi < 0 || bi >= n_box || beta >= Q || beta == 13 || !(q > 0.0 && q <= 1.0))
            return fail(LBM_ERR_INVALID_ARG, "link " + std::to_string(l) + " out of range");
        if (mask[bi] != 1) return fail(LBM_ERR_INVALID_ARG, "link " + std::to_string(l) + ": cell is not a plain fluid cell");
        const int x = (int)(bi % nx), y = (int)((bi / nx) % ny), z = (int)(bi / ((int64_t)nx * ny));
        if (shifted_fluid(x, y, z, beta, +1) >= 0)
            return fail(LBM_ERR_INVALID_ARG, "link " + std::to_string(l) + " does not point into a wall");
        lk.push_back({slot_of(x, y, z), {Q - 1 - beta, (float)q}});
    }
    std::sort(lk.begin(), lk.end(), [](const auto& a, const auto& b) {
        return a.first != b.first ? a.first < b.first : a.second.first < b.second.first;
    });
    int64_t n_bq = 0;
    for (size_t l = 0; l < lk.size(); ++l) {
        if (l > 0 && lk[l].first == lk[l - 1].first && lk[l].second.first == lk[l - 1].second.first)
            return fail(LBM_ERR_INVALID_ARG, "duplicate link");
        if (l == 0 || lk[l].first != lk[l - 1].first) ++n_bq;
    }
    // Packed link lists: each Bouzidi cell (in slot order) owns the entries [aux, aux + number of
    // its wall links) of the q list and of the twist side buffer, one per wall link in direction
    // order (q = 0 for a wall link without q: halfway bounce-back), so that the few links of a
    // cell share one or two sectors.
    std::vector<float> bq;
    for (size_t l = 0; l < lk.size();) {
        const int64_t s = lk[l].first;
        const uint32_t wmk = word[(size_t)s] & WORD_WALL_MASK;
        float qq[Q] = {};
        size_t e = l;
        for (; e < lk.size() && lk[e].first == s; ++e) {
            if (!((wmk >> lk[e].second.first) & 1u))
                return fail(LBM_ERR_INVALID_ARG, "a Bouzidi link does not cross a wall link of its cell");
            qq[lk[e].second.first] = lk[e].second.second;
        }
        if (bq.size() + Q >= ((size_t)1 << 31)) return fail(LBM_ERR_INVALID_ARG, "too many Bouzidi links");
        word[(size_t)s] |= (uint32_t)KIND_BOUZIDI << WORD_KIND_SHIFT;
        aux[(size_t)s] = (int32_t)bq.size();
        for (int i = 0; i < Q; ++i)
            if ((wmk >> i) & 1u) bq.push_back(qq[i]);
        l = e;
    }
    const int64_t n_blinks = (int64_t)bq.size();

    // ---------------------------------------------------------------- halo faces
    // face f = 2 axis + side (side 1: the high face); positions of a face run over the other two
    // axes, the lower one fastest.  halo_slot: the halo cell on the face; inner_slot: the fluid
    // cell one layer inside.  Only faces that hold halo cells get tables.
    std::vector<int32_t> halo_slot[6], inner_slot[6];
    int64_t face_area[6] = {0, 0, 0, 0, 0, 0};
    if (n_halo) {
        for (int f = 0; f < 6; ++f) {
            const int a = f / 2, side = f % 2;
            const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
            const int64_t area = (int64_t)n3[b] * n3[c];
            const int layer = side ? n3[a] - 1 : 0, inner = side ? n3[a] - 2 : 1;
            std::vector<int32_t> hs((size_t)area, -1), is((size_t)area, -1);
            bool any = false;
            // the halo layer and the layer inside it are independent: the neighbour's halo
            // holds a copy of the whole inner layer, wherever that layer is fluid, whatever
            // this side's halo holds at the same position (the two cross-sections differ
            // wherever a cut crosses a curved vessel)
            for (int v = 0; v < n3[c]; ++v)
                for (int u = 0; u < n3[b]; ++u) {
                    int p[3];
                    p[a] = layer;
                    p[b] = u;
                    p[c] = v;
                    const int64_t bi = p[0] + (int64_t)nx * (p[1] + (int64_t)ny * p[2]);
                    if (mask[bi] == 4) {
                        any = true;
                        hs[(size_t)(u + (int64_t)n3[b] * v)] = (int32_t)slot_of(p[0], p[1], p[2]);
                    }
                    if (n3[a] < 2) continue;
                    p[a] = inner;
                    const int64_t ii = p[0] + (int64_t)nx * (p[1] + (int64_t)ny * p[2]);
                    if (mask[ii] >= 1 && mask[ii] <= 3)
                        is[(size_t)(u + (int64_t)n3[b] * v)] = (int32_t)slot_of(p[0], p[1], p[2]);
                }
            if (any) {
                halo_slot[f].swap(hs);
                inner_slot[f].swap(is);
                face_area[f] = area;
            }
        }
    }

    // ---------------------------------------------------------------- device
    lbm_domain* D = new (std::nothrow) lbm_domain();
    static std::atomic<uint64_t> next_serial{1};
    if (D) D->serial = next_serial.fetch_add(1);
    if (!D) return fail(LBM_ERR_OOM, "host allocation failed");
    D->nx = nx;
    D->ny = ny;
    D->nz = nz;
    D->params = P;
    D->n_fluid = n_fluid;
    D->n_bricks = n_bricks;
    D->n_store_bricks = n_store;
    D->n_slots = n_slots;
    D->n_bq = n_bq;
    D->n_blinks = n_blinks;
    D->n_io = (int64_t)io_phi.size();
    D->n_wall = n_wall;
    D->stream = static_cast<cudaStream_t>(cuda_stream);
    D->alloc = alloc;
    D->release = release;
    D->alloc_ctx = alloc_ctx;
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, mask, (size_t)n_box);
    h = fnv1a(h, word.data(), word.size() * sizeof(uint32_t));
    h = fnv1a(h, bq.data(), bq.size() * sizeof(float));
    D->geometry_hash = h;

    lbm_status st = LBM_OK;
    int32_t* d_nbr = nullptr;
    int32_t* d_nb8 = nullptr;
    uint32_t* d_word = nullptr;
    float* d_s2 = nullptr;
    int32_t* d_aux = nullptr;
    float* d_bq = nullptr;
    float* d_io_phi = nullptr;
    int8_t* d_io_axis = nullptr;
    int8_t* d_io_sign = nullptr;
    if (!st) st = upload(D, &d_nbr, nbr, "brick neighbours");
    if (!st) st = upload(D, &d_nb8, nb8, "brick corner neighbours");
    if (!st) st = upload(D, &d_word, word, "cell words");
    if (!st) st = upload(D, &d_s2, s2_cell, "cell relaxation rates");
    if (!st) st = upload(D, &d_aux, aux, "aux index");
    if (!st) st = upload(D, &d_bq, bq, "Bouzidi q");
    if (!st) st = upload(D, &d_io_phi, io_phi, "inlet profile");
    if (!st) st = upload(D, &d_io_axis, io_axis, "open-boundary axis");
    if (!st) st = upload(D, &d_io_sign, io_sign, "open-boundary sign");
    if (!st) st = upload(D, &D->d_fl_slot, fl_slot, "fluid slots");
    if (!st) st = upload(D, &D->d_fl_box, fl_box, "fluid box indices");
    D->n_halo = n_halo;
    for (int f = 0; f < 6 && !st; ++f) {
        if (!face_area[f]) continue;
        D->face_area[f] = face_area[f];
        st = upload(D, &D->d_halo_slot[f], halo_slot[f], "halo slots");
        if (!st) st = upload(D, &D->d_inner_slot[f], inner_slot[f], "halo inner slots");
    }
    for (int k = 0; k < (twist ? 1 : 2) && !st; ++k) {
        D->d_pop[k] = D->dev_alloc(D->pop_bytes());
        if (!D->d_pop[k]) st = fail(LBM_ERR_OOM, "allocation failed: populations");
        else {
            cudaError_t e = cudaMemsetAsync(D->d_pop[k], 0, D->pop_bytes(), D->stream);
            if (e != cudaSuccess) st = cuda_fail(e, "clearing populations");
        }
    }
    if (!st && twist) {
        D->d_side = D->dev_alloc(D->side_bytes());
        if (!D->d_side) st = fail(LBM_ERR_OOM, "allocation failed: Bouzidi side buffer");
        else {
            cudaError_t e = cudaMemsetAsync(D->d_side, 0, D->side_bytes(), D->stream);
            if (e != cudaSuccess) st = cuda_fail(e, "clearing the side buffer");
        }
    }
    if (!st) {
        D->d_partials = static_cast<double*>(D->dev_alloc(sizeof(double) * 5 * (size_t)diagnostics_blocks(n_fluid)));
        D->d_diag = static_cast<lbm_diagnostics*>(D->dev_alloc(sizeof(lbm_diagnostics)));
        if (!D->d_partials || !D->d_diag) st = fail(LBM_ERR_OOM, "allocation failed: diagnostics");
    }
    if (!st) {
        cudaError_t e = cudaStreamSynchronize(D->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "uploading the domain");
    }
    if (st) {
        cudaStreamSynchronize(D->stream);
        D->release_all();
        delete D;
        return st;
    }
    DomainView& v = D->view;
    v.n_slots = n_slots;
    v.n_bricks = n_bricks;
    v.nbr = d_nbr;
    v.nb8 = d_nb8;
    v.side = D->d_side;
    v.word = d_word;
    v.s2_cell = d_s2;
    v.aux = d_aux;
    v.bq = d_bq;
    v.n_bq = std::max<int64_t>(n_blinks, 1);
    v.io_phi = d_io_phi;
    v.io_axis = d_io_axis;
    v.io_sign = d_io_sign;
    v.n_io = D->n_io;
    D->cur = 0;
    D->time = 0;
    *out = D;
    return LBM_OK;
}

lbm_status lbm_set_inlet_waveform(lbm_domain* D, const double* a, const double* b, int32_t n_harm,
                                  double period_steps, double u_peak)
{
    g_last_error.clear();
    if (!D || !a || (n_harm > 0 && !b)) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (n_harm < 0 || n_harm > 15) return fail(LBM_ERR_INVALID_ARG, "n_harm must be in 0..15");
    if (!(period_steps >= 1.0) || period_steps > 16777216.0 || period_steps != std::floor(period_steps))
        return fail(LBM_ERR_INVALID_ARG, "period_steps must be a positive integer <= 2^24");
    if (!std::isfinite(u_peak)) return fail(LBM_ERR_INVALID_ARG, "u_peak must be finite");
    const int64_t P = (int64_t)period_steps;
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<double> s((size_t)P);
    double smax = -INFINITY;
    for (int64_t t = 0; t < P; ++t) {
        double v = a[0];
        for (int k = 1; k <= n_harm; ++k) {
            const double ph = two_pi * k * (double)t / period_steps;
            v += a[k] * std::cos(ph) + b[k - 1] * std::sin(ph);
        }
        s[(size_t)t] = v;
        smax = std::max(smax, v);
    }
    if (!(smax > 0.0)) return fail(LBM_ERR_INVALID_ARG, "the waveform's maximum must be positive");
    D->wave.resize((size_t)P);
    for (int64_t t = 0; t < P; ++t) D->wave[(size_t)t] = (float)(u_peak * s[(size_t)t] / smax);
    D->wave_a.assign(a, a + n_harm + 1);
    D->wave_b.assign(b ? b : a, b ? b + n_harm : a);
    D->wave_period = period_steps;
    D->wave_peak = u_peak;
    D->has_wave = true;
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_domain* D, const float* rho, const float* u, int32_t device_ptrs)
{
    g_last_error.clear();
    if (!D || !rho || !u) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    const int64_t n_box = (int64_t)D->nx * D->ny * D->nz;
    const float* dr = rho;
    const float* du = u;
    float* stage = nullptr;
    if (!device_ptrs) {
        stage = static_cast<float*>(D->dev_alloc(sizeof(float) * 4 * (size_t)n_box));
        if (!stage) return fail(LBM_ERR_OOM, "allocation failed: staging");
        cudaError_t e = cudaMemcpyAsync(stage, rho, sizeof(float) * n_box, cudaMemcpyHostToDevice, D->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(stage + n_box, u, sizeof(float) * 3 * n_box, cudaMemcpyHostToDevice, D->stream);
        if (e != cudaSuccess) return cuda_fail(e, "uploading fields");
        dr = stage;
        du = stage + n_box;
    }
    // the previous level's parity decides where the twist keeps each population
    const int parity_prev = (int)((D->time + 1) & 1);
    cudaError_t e = launchers(D->params.storage)
                        .init_equilibrium(D->params.scheme, D->view, D->src(), parity_prev, D->d_fl_slot, D->d_fl_box,
                                          D->n_fluid, dr, du, n_box, D->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    if (stage) {
        e = cudaStreamSynchronize(D->stream);
        D->dev_free(stage, sizeof(float) * 4 * (size_t)n_box);
        if (e != cudaSuccess) return cuda_fail(e, "init");
    }
    return LBM_OK;
}

lbm_status lbm_step(lbm_domain* D, int64_t n)
{
    NvtxRange nvtx_range("lbm_step");
    g_last_error.clear();
    if (!D) return fail(LBM_ERR_INVALID_ARG, "NULL domain");
    if (n < 0) return fail(LBM_ERR_INVALID_ARG, "n must be >= 0");
    for (int64_t k = 0; k < n; ++k) {
        const LevelArgs a = D->level_args(D->time);
        cudaError_t e = launchers(D->params.storage)
                            .step(D->params.scheme, D->launch_config, D->view, D->src(), D->dst(), a, D->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel");
        if (!D->twist()) D->cur = 1 - D->cur;
        D->time += 1;
    }
    return LBM_OK;
}

lbm_status lbm_set_launch_config(lbm_domain* D, int32_t config)
{
    g_last_error.clear();
    if (!D) return fail(LBM_ERR_INVALID_ARG, "NULL domain");
    if (config < 0 || config >= N_LAUNCH_CONFIGS) return fail(LBM_ERR_INVALID_ARG, "launch config out of range");
    D->launch_config = config;
    return LBM_OK;
}

// Whether a launch configuration has its own kernel for this domain (otherwise the launcher
// falls back to another configuration, which the autotuner then need not time again).
static bool config_applies(const lbm_domain* D, int c)
{
    const bool twist = D->params.scheme == LBM_SCHEME_ESOTERIC;
    if (c == 5) return twist && D->params.storage == LBM_STORE_FP32;
    if (c == 6 || c == 7) return twist && D->level_args(0).coll == COLL_CHM_FAST;
    return true;
}

lbm_status lbm_autotune(lbm_domain* D, int32_t trial_steps, int32_t* best_config, float* ms_per_step)
{
    NvtxRange nvtx_range("lbm_autotune");
    g_last_error.clear();
    if (!D || trial_steps < 1) return fail(LBM_ERR_INVALID_ARG, "bad arguments");
    if (D->n_bricks == 0) {
        if (best_config) *best_config = D->launch_config;
        return LBM_OK;
    }
    // The state is kept: each configuration runs from a copy of the current populations (and
    // side buffer), and the copy is restored at the end.
    const size_t pb = D->pop_bytes(), sb = D->twist() ? D->side_bytes() : 0;
    unsigned char* keep = static_cast<unsigned char*>(D->dev_alloc(pb + sb));
    if (!keep) return fail(LBM_ERR_OOM, "allocation failed: autotune copy");
    cudaError_t e = cudaMemcpyAsync(keep, D->src(), pb, cudaMemcpyDeviceToDevice, D->stream);
    if (e == cudaSuccess && sb) e = cudaMemcpyAsync(keep + pb, D->d_side, sb, cudaMemcpyDeviceToDevice, D->stream);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const Launchers& L = launchers(D->params.storage);
    int best = D->launch_config;
    float best_ms = INFINITY;
    for (int c = 0; c < N_LAUNCH_CONFIGS && e == cudaSuccess; ++c) {
        if (!config_applies(D, c)) {
            if (ms_per_step) ms_per_step[c] = -1.0f;
            continue;
        }
        // one untimed step, then trial_steps timed steps, with the level arguments of the
        // domain's next levels (parity alternates as in a real run)
        int cur = D->cur;
        for (int k = 0; k <= trial_steps && e == cudaSuccess; ++k) {
            if (k == 1) e = cudaEventRecord(t0, D->stream);
            if (e != cudaSuccess) break;
            const LevelArgs a = D->level_args(D->time + k);
            void* src = D->twist() ? D->d_pop[0] : D->d_pop[cur];
            void* dst = D->twist() ? D->d_pop[0] : D->d_pop[1 - cur];
            e = L.step(D->params.scheme, c, D->view, src, dst, a, D->stream);
            cur = 1 - cur;
        }
        if (e == cudaSuccess) e = cudaEventRecord(t1, D->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        ms /= (float)trial_steps;
        if (ms_per_step) ms_per_step[c] = ms;
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
        // restore the state for the next configuration
        if (e == cudaSuccess) e = cudaMemcpyAsync(D->src(), keep, pb, cudaMemcpyDeviceToDevice, D->stream);
        if (e == cudaSuccess && sb) e = cudaMemcpyAsync(D->d_side, keep + pb, sb, cudaMemcpyDeviceToDevice, D->stream);
    }
    cudaError_t e2 = cudaStreamSynchronize(D->stream);
    if (e == cudaSuccess) e = e2;
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    D->dev_free(keep, pb + sb);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    D->launch_config = best;
    if (best_config) *best_config = best;
    return LBM_OK;
}

lbm_status lbm_get_macroscopic(lbm_domain* D, float* rho, float* u, int32_t dense, int32_t device_ptrs)
{
    NvtxRange nvtx_range("lbm_get_macroscopic");
    g_last_error.clear();
    if (!D || !rho || !u) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    const int64_t n_out = dense ? (int64_t)D->nx * D->ny * D->nz : D->n_fluid;
    const LevelArgs a = D->level_args(D->time);
    float* dr = rho;
    float* du = u;
    float* stage = nullptr;
    const size_t bytes = sizeof(float) * 4 * (size_t)std::max<int64_t>(n_out, 1);
    if (!device_ptrs) {
        stage = static_cast<float*>(D->dev_alloc(bytes));
        if (!stage) return fail(LBM_ERR_OOM, "allocation failed: staging");
        dr = stage;
        du = stage + n_out;
    }
    cudaError_t e = cudaSuccess;
    if (dense) e = cudaMemsetAsync(dr, 0, sizeof(float) * n_out, D->stream);
    if (dense && e == cudaSuccess) e = cudaMemsetAsync(du, 0, sizeof(float) * 3 * n_out, D->stream);
    if (e == cudaSuccess)
        e = launchers(D->params.storage)
                .macroscopic(D->params.scheme, D->view, D->src(), a, D->d_fl_slot, D->d_fl_box, D->n_fluid, dense, dr,
                             du, n_out, D->stream);
    if (stage) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(rho, dr, sizeof(float) * n_out, cudaMemcpyDeviceToHost, D->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, du, sizeof(float) * 3 * n_out, cudaMemcpyDeviceToHost, D->stream);
        cudaError_t e2 = cudaStreamSynchronize(D->stream);
        if (e == cudaSuccess) e = e2;
        D->dev_free(stage, bytes);
    }
    if (e != cudaSuccess) return cuda_fail(e, "macroscopic export");
    return LBM_OK;
}

lbm_status lbm_mean_reset(lbm_domain* D)
{
    g_last_error.clear();
    if (!D) return fail(LBM_ERR_INVALID_ARG, "NULL domain");
    const size_t bytes = sizeof(Sum4) * (size_t)std::max<int64_t>(D->n_fluid, 1);
    if (!D->d_mean) {
        D->d_mean = static_cast<Sum4*>(D->dev_alloc(bytes));
        if (!D->d_mean) return fail(LBM_ERR_OOM, "allocation failed: running means");
    }
    cudaError_t e = cudaMemsetAsync(D->d_mean, 0, bytes, D->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the running means");
    D->n_mean = 0;
    return LBM_OK;
}

lbm_status lbm_mean_sample(lbm_domain* D)
{
    g_last_error.clear();
    if (!D) return fail(LBM_ERR_INVALID_ARG, "NULL domain");
    if (!D->d_mean) return fail(LBM_ERR_STATE, "lbm_mean_reset was not called");
    const LevelArgs a = D->level_args(D->time);
    cudaError_t e = launchers(D->params.storage)
                        .mean_sample(D->params.scheme, D->view, D->src(), a, D->d_fl_slot, D->n_fluid, D->d_mean,
                                     D->stream);
    if (e != cudaSuccess) return cuda_fail(e, "running-mean sample");
    ++D->n_mean;
    return LBM_OK;
}

lbm_status lbm_mean_get(lbm_domain* D, float* rho, float* u, int32_t dense, int32_t device_ptrs, int64_t* n_samples)
{
    g_last_error.clear();
    if (!D || !rho || !u) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (!D->d_mean || D->n_mean == 0) return fail(LBM_ERR_STATE, "no samples since lbm_mean_reset");
    if (n_samples) *n_samples = D->n_mean;
    const int64_t n_out = dense ? (int64_t)D->nx * D->ny * D->nz : D->n_fluid;
    float* dr = rho;
    float* du = u;
    float* stage = nullptr;
    const size_t bytes = sizeof(float) * 4 * (size_t)std::max<int64_t>(n_out, 1);
    if (!device_ptrs) {
        stage = static_cast<float*>(D->dev_alloc(bytes));
        if (!stage) return fail(LBM_ERR_OOM, "allocation failed: staging");
        dr = stage;
        du = stage + n_out;
    }
    cudaError_t e = cudaSuccess;
    if (dense) e = cudaMemsetAsync(dr, 0, sizeof(float) * n_out, D->stream);
    if (dense && e == cudaSuccess) e = cudaMemsetAsync(du, 0, sizeof(float) * 3 * n_out, D->stream);
    if (e == cudaSuccess) e = launch_mean_out(D->d_mean, D->d_fl_box, D->n_fluid, D->n_mean, dense, dr, du, n_out, D->stream);
    if (stage) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(rho, dr, sizeof(float) * n_out, cudaMemcpyDeviceToHost, D->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, du, sizeof(float) * 3 * n_out, cudaMemcpyDeviceToHost, D->stream);
        cudaError_t e2 = cudaStreamSynchronize(D->stream);
        if (e == cudaSuccess) e = e2;
        D->dev_free(stage, bytes);
    }
    if (e != cudaSuccess) return cuda_fail(e, "running-mean export");
    return LBM_OK;
}

lbm_status lbm_probe(lbm_domain* D, const int64_t* fluid_index, int32_t n, float* out, int32_t device_ptrs)
{
    g_last_error.clear();
    if (!D || n < 0 || (n > 0 && (!fluid_index || !out))) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return LBM_OK;
    if (!device_ptrs)
        for (int32_t p = 0; p < n; ++p)
            if (fluid_index[p] < 0 || fluid_index[p] >= D->n_fluid)
                return fail(LBM_ERR_INVALID_ARG, "probe index outside [0, n_fluid)");
    const LevelArgs a = D->level_args(D->time);
    const int64_t* di = fluid_index;
    float4* dout = reinterpret_cast<float4*>(out);
    void* stage = nullptr;
    const size_t bytes = (sizeof(int64_t) + sizeof(float4)) * (size_t)n;
    cudaError_t e = cudaSuccess;
    if (!device_ptrs) {
        stage = D->dev_alloc(bytes);
        if (!stage) return fail(LBM_ERR_OOM, "allocation failed: staging");
        dout = static_cast<float4*>(stage);
        di = reinterpret_cast<const int64_t*>(static_cast<char*>(stage) + sizeof(float4) * (size_t)n);
        e = cudaMemcpyAsync(const_cast<int64_t*>(di), fluid_index, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice,
                            D->stream);
    }
    if (e == cudaSuccess)
        e = launchers(D->params.storage)
                .probe(D->params.scheme, D->view, D->src(), a, D->d_fl_slot, D->n_fluid, di, n, dout, D->stream);
    if (stage) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToHost, D->stream);
        cudaError_t e2 = cudaStreamSynchronize(D->stream);
        if (e == cudaSuccess) e = e2;
        D->dev_free(stage, bytes);
    }
    if (e != cudaSuccess) return cuda_fail(e, "probe");
    return LBM_OK;
}

}  // extern "C"

namespace lbm {
cudaError_t enqueue_macroscopic_dense(lbm_domain* D, float* rho, float* u, bool clear)
{
    const int64_t n_box = (int64_t)D->nx * D->ny * D->nz;
    cudaError_t e = cudaSuccess;
    if (clear) e = cudaMemsetAsync(rho, 0, sizeof(float) * n_box, D->stream);
    if (clear && e == cudaSuccess) e = cudaMemsetAsync(u, 0, sizeof(float) * 3 * n_box, D->stream);
    if (e != cudaSuccess) return e;
    return launchers(D->params.storage)
        .macroscopic(D->params.scheme, D->view, D->src(), D->level_args(D->time), D->d_fl_slot, D->d_fl_box,
                     D->n_fluid, 1, rho, u, n_box, D->stream);
}

cudaError_t enqueue_velocity_correction(lbm_domain* D, const float* rho, const float* u, const float* du)
{
    const int64_t n_box = (int64_t)D->nx * D->ny * D->nz;
    return launchers(D->params.storage)
        .apply_du(D->params.scheme, D->view, D->src(), (int)((D->time + 1) & 1), D->d_fl_slot, D->d_fl_box,
                  D->n_fluid, rho, u, du, n_box, D->stream);
}
}  // namespace lbm

extern "C" {

lbm_status lbm_apply_velocity_correction(lbm_domain* D, const float* du, int32_t device_ptrs)
{
    NvtxRange nvtx_range("lbm_apply_velocity_correction");
    g_last_error.clear();
    if (!D || !du) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    const int64_t n_box = (int64_t)D->nx * D->ny * D->nz;
    // one staging buffer per domain, kept: the correction runs every few dozen steps, and the
    // work of successive calls is ordered on the domain's stream
    if (!D->d_corr_stage) {
        D->d_corr_stage = static_cast<float*>(D->dev_alloc(sizeof(float) * 7 * (size_t)std::max<int64_t>(n_box, 1)));
        if (!D->d_corr_stage) return fail(LBM_ERR_OOM, "allocation failed: staging");
    }
    float* stage = D->d_corr_stage;
    float* rho = stage;
    float* u = stage + n_box;
    const float* dd = du;
    cudaError_t e = cudaSuccess;
    if (!device_ptrs) {
        e = cudaMemcpyAsync(stage + 4 * n_box, du, sizeof(float) * 3 * n_box, cudaMemcpyHostToDevice, D->stream);
        dd = stage + 4 * n_box;
    }
    const LevelArgs a = D->level_args(D->time);
    const Launchers& L = launchers(D->params.storage);
    if (e == cudaSuccess)
        e = L.macroscopic(D->params.scheme, D->view, D->src(), a, D->d_fl_slot, D->d_fl_box, D->n_fluid, 1, rho, u,
                          n_box, D->stream);
    if (e == cudaSuccess) e = enqueue_velocity_correction(D, rho, u, dd);
    if (!device_ptrs) {  // the host array may be reused as soon as the call returns
        cudaError_t e2 = cudaStreamSynchronize(D->stream);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail(e, "velocity correction");
    return LBM_OK;
}

lbm_status lbm_get_diagnostics(lbm_domain* D, lbm_diagnostics* out)
{
    NvtxRange nvtx_range("lbm_get_diagnostics");
    g_last_error.clear();
    if (!D || !out) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    const LevelArgs a = D->level_args(D->time);
    cudaError_t e = launchers(D->params.storage)
                        .diagnostics(D->params.scheme, D->view, D->src(), a, D->d_fl_slot, D->n_fluid, D->d_partials,
                                     D->stream);
    if (e == cudaSuccess) e = launch_diagnostics_final(D->d_partials, diagnostics_blocks(D->n_fluid), D->d_diag, D->stream);
    lbm_diagnostics h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, D->d_diag, sizeof(h), cudaMemcpyDeviceToHost, D->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(D->stream);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics");
    if (lbm_status ds = debug_status(D->params.storage)) return ds;
    h.time = D->time;
    *out = h;
    if (h.n_nonfinite > 0) return fail(LBM_ERR_UNSTABLE, "non-finite populations in " + std::to_string(h.n_nonfinite) + " cells");
    return LBM_OK;
}

lbm_status lbm_get_info(const lbm_domain* D, lbm_info* out)
{
    g_last_error.clear();
    if (!D || !out) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    lbm_info I{};
    I.nx = D->nx;
    I.ny = D->ny;
    I.nz = D->nz;
    I.n_fluid = D->n_fluid;
    I.n_bricks = D->n_bricks;
    I.n_slots = D->n_slots;
    I.n_wall_cells = D->n_wall;
    I.n_bouzidi_cells = D->n_bq;
    I.n_open_cells = D->n_io;
    I.time = D->time;
    I.storage = D->params.storage;
    I.bytes_per_value = D->bytes_per_value();
    I.device_bytes = D->device_bytes;
    I.launch_config = D->launch_config;
    I.scheme = D->params.scheme;
    I.n_store_bricks = D->n_store_bricks;
    I.n_halo = D->n_halo;
    *out = I;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_domain* D)
{
    g_last_error.clear();
    if (!D) return fail(LBM_ERR_INVALID_ARG, "NULL domain");
    cudaError_t e = cudaStreamSynchronize(D->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    return debug_status(D->params.storage);
}

// ------------------------------------------------------------------------ checkpoints
namespace {
struct CheckpointHeader {
    char magic[8];
    uint32_t version;
    int32_t nx, ny, nz, storage;
    int64_t n_slots, time;
    uint64_t geometry_hash;
    lbm_params params;
    int32_t has_wave, n_harm;
    double wave_period, wave_peak;
};
const char kMagic[8] = {'L', 'B', 'M', 'G', 'B', '3', '0', '0'};
}  // namespace

lbm_status lbm_save_state(lbm_domain* D, const char* path)
{
    g_last_error.clear();
    if (!D || !path) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    const size_t sb = D->twist() ? D->side_bytes() : 0;
    std::vector<unsigned char> buf(D->pop_bytes() + sb);
    cudaError_t e = cudaMemcpyAsync(buf.data(), D->src(), D->pop_bytes(), cudaMemcpyDeviceToHost, D->stream);
    if (e == cudaSuccess && sb)
        e = cudaMemcpyAsync(buf.data() + D->pop_bytes(), D->d_side, sb, cudaMemcpyDeviceToHost, D->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(D->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading populations");
    CheckpointHeader H{};
    std::memcpy(H.magic, kMagic, 8);
    H.version = 3;
    H.nx = D->nx;
    H.ny = D->ny;
    H.nz = D->nz;
    H.storage = D->params.storage;
    H.n_slots = D->n_slots;
    H.time = D->time;
    H.geometry_hash = D->geometry_hash;
    H.params = D->params;
    H.has_wave = D->has_wave ? 1 : 0;
    H.n_harm = D->has_wave ? (int32_t)D->wave_a.size() - 1 : 0;
    H.wave_period = D->wave_period;
    H.wave_peak = D->wave_peak;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&H, sizeof(H), 1, f) == 1;
    if (ok && H.has_wave) {
        ok = std::fwrite(D->wave_a.data(), sizeof(double), D->wave_a.size(), f) == D->wave_a.size();
        if (ok && H.n_harm > 0) ok = std::fwrite(D->wave_b.data(), sizeof(double), D->wave_b.size(), f) == D->wave_b.size();
    }
    if (ok) ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(LBM_ERR_IO, std::string("write failed: ") + path);
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_domain* D, const char* path)
{
    g_last_error.clear();
    if (!D || !path) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    CheckpointHeader H{};
    bool ok = std::fread(&H, sizeof(H), 1, f) == 1;
    if (!ok || std::memcmp(H.magic, kMagic, 8) != 0 || H.version != 3) {
        std::fclose(f);
        return fail(LBM_ERR_IO, "not a checkpoint of this library");
    }
    if (H.nx != D->nx || H.ny != D->ny || H.nz != D->nz || H.storage != D->params.storage ||
        H.params.scheme != D->params.scheme || H.n_slots != D->n_slots || H.geometry_hash != D->geometry_hash) {
        std::fclose(f);
        return fail(LBM_ERR_IO, "checkpoint does not match this domain's geometry or storage");
    }
    std::vector<double> wa, wb;
    if (H.has_wave) {
        if (H.n_harm < 0 || H.n_harm > 15) {
            std::fclose(f);
            return fail(LBM_ERR_IO, "corrupt checkpoint");
        }
        wa.resize((size_t)H.n_harm + 1);
        wb.resize((size_t)H.n_harm);
        ok = std::fread(wa.data(), sizeof(double), wa.size(), f) == wa.size();
        if (ok && H.n_harm > 0) ok = std::fread(wb.data(), sizeof(double), wb.size(), f) == wb.size();
    }
    const size_t sb = D->twist() ? D->side_bytes() : 0;
    std::vector<unsigned char> buf(D->pop_bytes() + sb);
    if (ok) ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return fail(LBM_ERR_IO, "truncated checkpoint");
    if (lbm_status s = check_params(H.params)) return s;
    cudaError_t e = cudaMemcpyAsync(D->src(), buf.data(), D->pop_bytes(), cudaMemcpyHostToDevice, D->stream);
    if (e == cudaSuccess && sb)
        e = cudaMemcpyAsync(D->d_side, buf.data() + D->pop_bytes(), sb, cudaMemcpyHostToDevice, D->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(D->stream);
    if (e != cudaSuccess) return cuda_fail(e, "writing populations");
    D->params = H.params;
    D->time = H.time;
    if (H.has_wave) {
        lbm_status s = lbm_set_inlet_waveform(D, wa.data(), wb.empty() ? nullptr : wb.data(), H.n_harm,
                                              H.wave_period, H.wave_peak);
        if (s) return s;
    } else {
        D->has_wave = false;
        D->wave.clear();
    }
    return LBM_OK;
}

lbm_status lbm_halo_size(const lbm_domain* D, int32_t face, int64_t* values)
{
    g_last_error.clear();
    if (!D || !values) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (face < 0 || face > 5) return fail(LBM_ERR_INVALID_ARG, "face must be 0..5");
    *values = 9 * D->face_area[face];
    return LBM_OK;
}

static lbm_status halo_copy(lbm_domain* D, int32_t face, void* buf, bool pack)
{
    NvtxRange nvtx_range("lbm_halo_copy");
    g_last_error.clear();
    if (!D || !buf) return fail(LBM_ERR_INVALID_ARG, "NULL argument");
    if (face < 0 || face > 5) return fail(LBM_ERR_INVALID_ARG, "face must be 0..5");
    if (!D->face_area[face]) return fail(LBM_ERR_INVALID_ARG, "the face has no halo layer");
    // pack: the populations leaving through the face (c . n_out = +1) from the layer inside the
    // halo; unpack: the populations entering through it (c . n_out = -1) into the halo layer.
    // Both list the directions with c_axis = (face high ? +1 : -1) for pack and the opposite for
    // unpack, in increasing i -- the same list on the two sides of a cut.
    const int a = face / 2, side = face % 2;
    const int c_out = side ? +1 : -1;
    const int want = pack ? c_out : -c_out;
    HaloDirs dirs{};
    int k = 0;
    for (int i = 0; i < Q; ++i) {
        const int ci = a == 0 ? cx_of(i) : a == 1 ? cy_of(i) : cz_of(i);
        if (ci == want) dirs.d[k++] = (int8_t)i;
    }
    cudaError_t e = launch_halo_copy(D->bytes_per_value(), pack, D->src(), D->view.n_slots,
                                     pack ? D->d_inner_slot[face] : D->d_halo_slot[face], D->face_area[face], dirs,
                                     buf, D->stream);
    if (e != cudaSuccess) return cuda_fail(e, pack ? "halo pack" : "halo unpack");
    return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_domain* D, int32_t face, void* buf) { return halo_copy(D, face, buf, true); }

lbm_status lbm_halo_unpack(lbm_domain* D, int32_t face, const void* buf)
{
    return halo_copy(D, face, const_cast<void*>(buf), false);
}

void lbm_destroy(lbm_domain* D)
{
    if (!D) return;
    cudaStreamSynchronize(D->stream);
    D->release_all();
    delete D;
}

}  // extern "C"

// ------------------------------------------------------------------------ batches
struct lbm_batch {
    std::vector<lbm_domain*> doms;
    int storage = 0;
    int coll = COLL_CHM_FAST;
    int launch_config = DEFAULT_LAUNCH_CONFIG;
    int graph_steps = 0;
    int64_t total_bricks = 0, total_fluid = 0;
    cudaStream_t stream = nullptr;       // private non-blocking stream: work and graph capture
    cudaStream_t user_stream = nullptr;  // the caller's stream, ordered before and after
    lbm_domain* owner = nullptr;  // its allocator serves the batch's buffers
    BatchEntry* d_ent = nullptr;
    int64_t* d_start = nullptr;
    LevelArgs* d_args = nullptr;  // [graph_steps][n]
    LevelArgs* h_args = nullptr;  // pinned mirror
    size_t args_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    int exec_config = -1;
    int exec_parity = -2;  // common parity of the captured chunk's first step (-1: mixed)
    bool exec_persistent = false;
    cudaEvent_t ev = nullptr;
    // persistent mode: one cooperative launch per chunk, a bounded grid barrier between steps
    bool persistent = false;
    uint64_t limit_ns = 1000000000ull;
    GridBarrier* d_bar = nullptr;
    unsigned int* h_fail = nullptr;  // pinned: the barrier's fail word after the last chunk

    int n() const { return (int)doms.size(); }
    // the parity all domains have at step k of the argument table, or -1 if they differ
    int common_parity(int k) const
    {
        const int p = h_args[(size_t)k * n()].parity;
        for (int d = 1; d < n(); ++d)
            if (h_args[(size_t)k * n() + d].parity != p) return -1;
        return p;
    }
    void fill_args(int steps)
    {
        for (int k = 0; k < steps; ++k)
            for (int d = 0; d < n(); ++d) h_args[(size_t)k * n() + d] = doms[(size_t)d]->level_args(doms[(size_t)d]->time + k);
    }
    // orders the batch's stream after, or before, the work of every member domain's stream
    cudaError_t join_from_domains()
    {
        cudaError_t e = cudaEventRecord(ev, user_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev, 0);
        for (lbm_domain* D : doms) {
            if (e != cudaSuccess) break;
            e = cudaEventRecord(ev, D->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev, 0);
        }
        return e;
    }
    cudaError_t join_to_domains()
    {
        cudaError_t e = cudaEventRecord(ev, stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(user_stream, ev, 0);
        for (lbm_domain* D : doms) {
            if (e != cudaSuccess) break;
            e = cudaStreamWaitEvent(D->stream, ev, 0);
        }
        return e;
    }
    cudaError_t enqueue_steps(int steps, int config)
    {
        cudaError_t e = cudaMemcpyAsync(d_args, h_args, sizeof(LevelArgs) * (size_t)steps * n(), cudaMemcpyHostToDevice,
                                        stream);
        const Launchers& L = launchers(storage);
        if (persistent) {
            // the barrier word and the per-step ticket counters that follow it
            if (e == cudaSuccess)
                e = cudaMemsetAsync(d_bar, 0, sizeof(GridBarrier) + sizeof(unsigned int) * (size_t)steps, stream);
            if (e == cudaSuccess)
                e = L.step_batch_persistent(d_ent, d_start, n(), total_bricks, d_args, coll, common_parity(0), steps,
                                            d_bar, limit_ns, stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_fail, &d_bar->fail, sizeof(unsigned int), cudaMemcpyDeviceToHost, stream);
            return e;
        }
        for (int k = 0; k < steps && e == cudaSuccess; ++k)
            e = L.step_batch(config, d_ent, d_start, n(), total_bricks, d_args + (size_t)k * n(), coll,
                             common_parity(k), stream);
        return e;
    }
    cudaError_t capture()
    {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        e = enqueue_steps(graph_steps, launch_config);
        cudaError_t e2 = cudaStreamEndCapture(stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        exec_config = (e == cudaSuccess) ? launch_config : -1;
        exec_parity = (e == cudaSuccess) ? common_parity(0) : -2;
        exec_persistent = persistent;
        return e;
    }
    // a persistent chunk that has completed gave up at a barrier
    bool timed_out() const { return persistent && h_fail && *h_fail != 0u; }
    void release()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (ev) cudaEventDestroy(ev);
        if (stream) cudaStreamDestroy(stream);
        if (h_args) cudaFreeHost(h_args);
        if (h_fail) cudaFreeHost(h_fail);
        for (void* p : {(void*)d_ent, (void*)d_start, (void*)d_args, (void*)d_bar})
            if (p) owner->dev_free(p, 0);
    }
};

extern "C" {

lbm_status lbm_batch_create(lbm_domain* const* doms, int32_t n, int32_t graph_steps, void* cuda_stream,
                            lbm_batch** out)
{
    g_last_error.clear();
    if (!out) return fail(LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!doms || n < 1 || n > 4096) return fail(LBM_ERR_INVALID_ARG, "need 1..4096 domains");
    if (graph_steps < 1 || graph_steps > 4096) return fail(LBM_ERR_INVALID_ARG, "graph_steps must be in 1..4096");
    for (int d = 0; d < n; ++d) {
        if (!doms[d]) return fail(LBM_ERR_INVALID_ARG, "NULL domain in the batch");
        if (doms[d]->params.scheme != LBM_SCHEME_ESOTERIC)
            return fail(LBM_ERR_INVALID_ARG, "batched domains must use the esoteric-twist scheme");
        if (doms[d]->params.storage != doms[0]->params.storage)
            return fail(LBM_ERR_INVALID_ARG, "batched domains must share one storage precision");
        if (doms[d]->level_args(0).coll != doms[0]->level_args(0).coll)
            return fail(LBM_ERR_INVALID_ARG,
                        "batched domains must share one collision kernel (operator, and for CHM-MRT whether "
                        "all higher-order rates are 1)");
        for (int e = 0; e < d; ++e)
            if (doms[e] == doms[d]) return fail(LBM_ERR_INVALID_ARG, "a domain appears twice in the batch");
    }
    lbm_batch* B = new (std::nothrow) lbm_batch();
    if (!B) return fail(LBM_ERR_OOM, "host allocation failed");
    B->doms.assign(doms, doms + n);
    B->storage = doms[0]->params.storage;
    B->coll = doms[0]->level_args(0).coll;
    B->graph_steps = graph_steps;
    B->user_stream = static_cast<cudaStream_t>(cuda_stream);
    B->owner = doms[0];
    std::vector<BatchEntry> ent((size_t)n);
    std::vector<int64_t> start((size_t)n + 1, 0);
    for (int d = 0; d < n; ++d) {
        ent[(size_t)d].view = doms[d]->view;
        ent[(size_t)d].pop = doms[d]->d_pop[0];
        start[(size_t)d + 1] = start[(size_t)d] + doms[d]->n_bricks;
        B->total_fluid += doms[d]->n_fluid;
    }
    B->total_bricks = start[(size_t)n];
    B->args_bytes = sizeof(LevelArgs) * (size_t)graph_steps * (size_t)n;
    cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_args, B->args_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_fail, sizeof(unsigned int));
    if (e == cudaSuccess) *B->h_fail = 0u;
    lbm_status st = (e == cudaSuccess) ? LBM_OK : cuda_fail(e, "batch set-up");
    if (!st) {
        B->d_ent = static_cast<BatchEntry*>(B->owner->dev_alloc(sizeof(BatchEntry) * (size_t)n));
        B->d_start = static_cast<int64_t*>(B->owner->dev_alloc(sizeof(int64_t) * ((size_t)n + 1)));
        B->d_args = static_cast<LevelArgs*>(B->owner->dev_alloc(B->args_bytes));
        B->d_bar = static_cast<GridBarrier*>(
            B->owner->dev_alloc(sizeof(GridBarrier) + sizeof(unsigned int) * (size_t)graph_steps));
        if (!B->d_ent || !B->d_start || !B->d_args || !B->d_bar) st = fail(LBM_ERR_OOM, "allocation failed: batch tables");
    }
    if (!st) {
        e = cudaMemcpyAsync(B->d_ent, ent.data(), sizeof(BatchEntry) * ent.size(), cudaMemcpyHostToDevice, B->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B->d_start, start.data(), sizeof(int64_t) * start.size(), cudaMemcpyHostToDevice,
                                B->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
        // the domains' buffers were cleared / uploaded on their own streams
        for (int d = 0; d < n && e == cudaSuccess; ++d) e = cudaStreamSynchronize(doms[d]->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "uploading the batch tables");
    }
    if (st) {
        B->release();
        delete B;
        return st;
    }
    *out = B;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* B, int64_t n)
{
    NvtxRange nvtx_range("lbm_batch_step");
    g_last_error.clear();
    if (!B) return fail(LBM_ERR_INVALID_ARG, "NULL batch");
    if (n < 0) return fail(LBM_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return LBM_OK;
    cudaError_t e = B->join_from_domains();
    while (n > 0 && e == cudaSuccess) {
        const int k = (int)std::min<int64_t>(n, B->graph_steps);
        // the pinned argument table is reused: wait until the previous chunk has read it
        e = cudaStreamSynchronize(B->stream);
        if (e != cudaSuccess) break;
        if (B->timed_out()) {
            *B->h_fail = 0u;
            B->join_to_domains();
            return fail(LBM_ERR_TIMEOUT, "persistent batch: a grid barrier wait gave up; the members' populations "
                                         "are undefined");
        }
        B->fill_args(k);
        if (k == B->graph_steps) {
            // the captured kernels are specialised by parity: recapture if the chunk starts
            // with another one (an odd chunk length, or members stepped on their own)
            if (!B->exec || B->exec_config != B->launch_config || B->exec_parity != B->common_parity(0) ||
                B->exec_persistent != B->persistent)
                e = B->capture();
            if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, B->stream);
        } else {
            e = B->enqueue_steps(k, B->launch_config);
        }
        if (e == cudaSuccess)
            for (lbm_domain* D : B->doms) D->time += k;
        n -= k;
    }
    if (e == cudaSuccess) e = B->join_to_domains();
    if (e != cudaSuccess) return cuda_fail(e, "batch step");
    return LBM_OK;
}

lbm_status lbm_batch_set_persistent(lbm_batch* B, int32_t enable, double barrier_timeout_s)
{
    g_last_error.clear();
    if (!B) return fail(LBM_ERR_INVALID_ARG, "NULL batch");
    if (!(barrier_timeout_s > 0.0) || !(barrier_timeout_s <= 3600.0))
        return fail(LBM_ERR_INVALID_ARG, "barrier_timeout_s must be in (0, 3600]");
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch");
    B->persistent = enable != 0;
    B->limit_ns = (uint64_t)std::max(1.0, barrier_timeout_s * 1e9);
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* B)
{
    g_last_error.clear();
    if (!B) return fail(LBM_ERR_INVALID_ARG, "NULL batch");
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    if (B->timed_out()) {
        *B->h_fail = 0u;
        return fail(LBM_ERR_TIMEOUT, "persistent batch: a grid barrier wait gave up; the members' populations are "
                                     "undefined");
    }
    return LBM_OK;
}

lbm_status lbm_batch_set_launch_config(lbm_batch* B, int32_t config)
{
    g_last_error.clear();
    if (!B) return fail(LBM_ERR_INVALID_ARG, "NULL batch");
    if (config < 0 || config >= N_LAUNCH_CONFIGS) return fail(LBM_ERR_INVALID_ARG, "launch config out of range");
    B->launch_config = config;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* B, int32_t trial_steps, int32_t* best_config, float* ms_per_step)
{
    g_last_error.clear();
    if (!B || trial_steps < 1 || trial_steps > B->graph_steps)
        return fail(LBM_ERR_INVALID_ARG, "trial_steps must be in 1..graph_steps");
    // keep every member's populations and side buffer; run each configuration; restore
    std::vector<std::pair<void*, size_t>> keep;
    cudaError_t e = B->join_from_domains();
    lbm_status st = LBM_OK;
    for (lbm_domain* D : B->doms) {
        const size_t bytes = D->pop_bytes() + D->side_bytes();
        unsigned char* p = static_cast<unsigned char*>(B->owner->dev_alloc(bytes));
        if (!p) {
            st = fail(LBM_ERR_OOM, "allocation failed: batch autotune copy");
            break;
        }
        keep.push_back({p, bytes});
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, D->d_pop[0], D->pop_bytes(), cudaMemcpyDeviceToDevice, B->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p + D->pop_bytes(), D->d_side, D->side_bytes(), cudaMemcpyDeviceToDevice, B->stream);
    }
    const bool was_persistent = B->persistent;
    B->persistent = false;  // the trial times the one-launch-per-step configurations
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (!st && e == cudaSuccess) e = cudaEventCreate(&t0);
    if (!st && e == cudaSuccess) e = cudaEventCreate(&t1);
    int best = B->launch_config;
    float best_ms = INFINITY;
    if (!st && e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (!st && e == cudaSuccess) B->fill_args(trial_steps);
    // back to the kept populations and side buffers (stream-ordered copies)
    auto restore = [&]() {
        for (size_t d = 0; d < keep.size() && e == cudaSuccess; ++d) {
            lbm_domain* D = B->doms[d];
            unsigned char* p = static_cast<unsigned char*>(keep[d].first);
            e = cudaMemcpyAsync(D->d_pop[0], p, D->pop_bytes(), cudaMemcpyDeviceToDevice, B->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(D->d_side, p + D->pop_bytes(), D->side_bytes(), cudaMemcpyDeviceToDevice, B->stream);
        }
    };
    for (int c = 0; c < N_LAUNCH_CONFIGS && !st && e == cudaSuccess; ++c) {
        if (c >= 5) {  // the batched kernel has the one-cell configurations 0-4 only
            if (ms_per_step) ms_per_step[c] = -1.0f;
            continue;
        }
        // one untimed step, then the trial from the kept state again, so that the timed steps
        // run the levels of the argument table in order (parity alternating as in a real run)
        e = B->enqueue_steps(1, c);
        restore();
        if (e == cudaSuccess) e = cudaEventRecord(t0, B->stream);
        if (e == cudaSuccess) e = B->enqueue_steps(trial_steps, c);
        if (e == cudaSuccess) e = cudaEventRecord(t1, B->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        ms /= (float)trial_steps;
        if (ms_per_step) ms_per_step[c] = ms;
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
        restore();
    }
    cudaError_t e2 = cudaStreamSynchronize(B->stream);
    if (e == cudaSuccess) e = e2;
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    for (auto& k : keep) B->owner->dev_free(k.first, k.second);
    B->persistent = was_persistent;
    if (e == cudaSuccess) e = B->join_to_domains();
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
    B->launch_config = best;
    if (best_config) *best_config = best;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* B)
{
    if (!B) return;
    cudaStreamSynchronize(B->stream);
    B->release();
    delete B;
}

}  // extern "C"

namespace lbm {

bool domain_access(const lbm_domain* D, DomainAccess* out)
{
    if (!D || !out) return false;
    out->storage = D->params.storage;
    out->scheme = D->params.scheme;
    out->view = &D->view;
    out->src = D->src();
    out->args = D->level_args(D->time);
    out->fl_slot = D->d_fl_slot;
    out->n_fluid = D->n_fluid;
    out->time = D->time;
    out->stream = D->stream;
    out->serial = D->serial;
    return true;
}

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

}  // namespace lbm
