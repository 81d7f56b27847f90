// lbm_api.cu -- the C ABI declared in include/lbm.h: handle life cycle,
// packed ragged layout of a batch, stepping, observables, field access,
// checkpoints.  All arithmetic of the method runs in the kernels of
// lbm_step.cu and lbm_aux.cu; this file only sizes, allocates, copies and
// launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbmk {
// store: 0 FP32, 1 FP16, 2 BF16 storage
cudaError_t launch_step_direct(const StepArgs &a, int ntiles, int tx,
                               int ty, int store, cudaStream_t s);
cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap *pop_maps,
                            const CUtensorMap *mask_maps,
                            const CUtensorMap *out_maps, const TileRec *sched,
                            int nslots, int grid, int tx, int ty, int store,
                            int *err, cudaStream_t s);
cudaError_t grid_step_tma(int tx, int ty, int store, int *grid);
int tma_box_x(int tx);
int tma_mask_box_x(int tx);
__global__ void k_unstream(const LatDesc *, int, const float *,
                           const uint8_t *, uint8_t, void *, bool);
__global__ void k_export(const LatDesc *, int, const void *, const uint8_t *,
                         const double *, long long, bool, float *, float *,
                         double *);
__global__ void k_settle(const LatDesc *, int, const void *, uint8_t *,
                         double *, LatState *, long long, bool);
__global__ void k_mask_agree(const LatDesc *, int, uint8_t *, long long);
__global__ void k_solid_mask(const LatDesc *, int, const uint8_t *, uint8_t,
                             uint8_t *);
__global__ void k_gather_inputs(const InPtrs *, int, const int64_t *, float *,
                                uint8_t *);
__global__ void k_mask_init_all(const LatDesc *, int, const int64_t *,
                                const int64_t *, const uint8_t *, uint8_t *);
__global__ void k_col_init_all(const LatDesc *, int, const int64_t *,
                               const int64_t *, const uint8_t *, int32_t *,
                               int16_t *, LatState *);
__global__ void k_init_rest_all(const LatDesc *, int, const int64_t *,
                                const int64_t *, const float *, const uint8_t *,
                                void *, bool);
__global__ void k_solid_mask_all(const LatDesc *, int, const int64_t *,
                                 const int64_t *, const uint8_t *, uint8_t,
                                 uint8_t *);
void launch_obs_columns(bool summed, int store, int nb, int ncols,
                        const LatDesc *desc, const int32_t *col_lat,
                        const int64_t *col_base, const void *fin,
                        const uint8_t *mask, const double *m, long long t,
                        ColObs *out, cudaStream_t s);
struct LbmObsDev;
__global__ void k_obs_reduce(const LatDesc *, const int64_t *,
                             const ColObs *, const int16_t *,
                             const LatState *, const double *, long long,
                             LbmObsDev *);
}  // namespace lbmk

using namespace lbmk;

static_assert(sizeof(lbm_obs) == 8 * 16 + 4 * 2 + 8, "lbm_obs layout");

struct lbm_handle {
    int count = 0;
    bool half = false;  // 16-bit storage (FP16 or BF16): the 15-word layout
    bool bf16 = false;  // its format
    // 0 FP32, 1 FP16, 2 BF16 (the step kernels' storage policy)
    int store() const { return half ? (bf16 ? 2 : 1) : 0; }
    // tile of the step kernel (LBM_TILE overrides, lbm_autotune picks per
    // workload); set by pick_tile
    int tx = 64, ty = 8;
    bool use_tma = true;
    std::vector<LatDesc> desc;
    std::vector<int64_t> col_base;   // first column of lattice l (all columns)
    std::vector<int64_t> in_off_host;  // first node of lattice l, unpadded (count + 1)
    int64_t ncols = 0;               // columns of all lattices
    int64_t nsec = 0;                // section columns of all lattices
    int ntiles = 0;
    int64_t pop_elems = 0, node_elems = 0;  // 32-bit words, mask bytes
    size_t max_nodes = 0;            // largest nx*ny
    // device
    LatDesc *d_desc = nullptr;
    int32_t *d_tile_lat = nullptr;
    int32_t *d_col_lat = nullptr;
    int64_t *d_col_base = nullptr;
    int64_t *d_in_off = nullptr;       // node then row prefixes, 2 (count + 1)
    int64_t total_rows = 0;
    uint8_t *d_masks = nullptr;        // all solid masks, unpadded (on first use)
    void *d_pop[2] = {nullptr, nullptr};
    uint8_t *d_mask = nullptr;
    double *d_m = nullptr;
    int32_t *d_col_fluid = nullptr;
    int16_t *d_wall0 = nullptr;
    LatState *d_st = nullptr;
    int64_t *d_step = nullptr;
    unsigned int *d_done = nullptr;
    ColObs *d_cols = nullptr;
    void *d_obs = nullptr;
    // [count][3] A, B and solute totals that the last launch of each
    // lbm_step call adds up, valid for step count sums_step
    double *d_sums = nullptr;
    int64_t sums_step = -1;
    float *d_canon = nullptr;      // [22][ny][nx] scratch of one lattice
    float *d_dens = nullptr;       // [3][ny][nx]
    double *d_dep = nullptr;       // [ny][nx]
    // [2 buffers][count] population maps over the ghost band for the tile
    // copies, then [2 buffers][count] over the lattice itself for the
    // output stores
    CUtensorMap *d_maps = nullptr;
    CUtensorMap *d_mask_maps = nullptr; // [count] mask maps
    TileRec *d_sched = nullptr;        // TMA kernel: tiles of each block
    int sched_grid = 0, sched_slots = 0;
    // kGraphSteps steps from cur == 0; [1]: the last launch sums the
    // lattice totals (the replay that ends an lbm_step call)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool use_graph = true;
    int stall_tx = 0;  // test hook, see pick_tile
    int *d_err = nullptr;              // kernel error flags
    int cur = 0;
    int64_t steps = 0;
    cudaStream_t own = nullptr, stream = nullptr;
    bool dead = false;
    std::string err;
};

static thread_local std::string g_create_err;

static lbm_status fail(lbm_handle *h, lbm_status st, const std::string &msg) {
    if (h) {
        h->err = msg;
        if (st == LBM_ECUDA) h->dead = true;
    } else {
        g_create_err = msg;
    }
    return st;
}

#define CK(h, call)                                                        \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess)                                             \
            return fail((h), LBM_ECUDA,                                    \
                        std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
static cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
}

static void free_all(lbm_handle *h) {
    void *ps[] = {h->d_desc, h->d_tile_lat, h->d_col_lat, h->d_col_base,
                  h->d_in_off, h->d_masks,
                  h->d_pop[0], h->d_pop[1],
                  h->d_mask, h->d_m, h->d_col_fluid, h->d_wall0, h->d_st,
                  h->d_step, h->d_done, h->d_cols, h->d_obs, h->d_canon,
                  h->d_dens, h->d_dep, h->d_maps, h->d_mask_maps, h->d_err,
                  h->d_sched, h->d_sums};
    for (void *p : ps)
        if (p) cudaFree(p);
    for (cudaGraphExec_t g : h->graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->own) cudaStreamDestroy(h->own);
}

static bool valid_params(const lbm_params &p, std::string &why) {
    if (!(p.tau_a > 0.5 && p.tau_b > 0.5 && p.tau_d > 0.5)) {
        why = "relaxation times must exceed 1/2";
        return false;
    }
    if (!(p.k_r >= 0.0) || !std::isfinite(p.k_r)) {
        why = "k_r must be finite and >= 0";
        return false;
    }
    if (!std::isfinite(p.g_coh) || !std::isfinite(p.g_ads) ||
        !std::isfinite(p.c_in) || !std::isfinite(p.body_force_x) ||
        std::isnan(p.m_threshold)) {
        why = "non-finite constant";
        return false;
    }
    // Deposit only grows, by the reaction: with a positive threshold a node
    // can only reach it in a step in which it reacts, which is where the
    // step kernel tests it.
    if (!(p.m_threshold > 0.0)) {
        why = "m_threshold must be > 0";
        return false;
    }
    if (p.precision != LBM_FP32 && p.precision != LBM_FP16 &&
        p.precision != LBM_BF16) {
        why = "unknown precision";
        return false;
    }
    return true;
}

// The address under which this device reads a caller's array, or null if
// it cannot (pageable host memory, another device's memory): pinned or
// registered host memory is mapped into the device's address space (its
// device pointer), managed memory and this device's memory are used as
// they are.
static const void *device_view(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    switch (a.type) {
    case cudaMemoryTypeHost:
        return a.devicePointer;
    case cudaMemoryTypeDevice:
        return a.device == dev ? a.devicePointer : nullptr;
    case cudaMemoryTypeManaged:
        return a.devicePointer ? a.devicePointer : p;
    default:
        return nullptr;
    }
}

static void pick_tile(lbm_handle *h) {
    // measured fastest on the batched sweep: 64 x 8 for FP32 storage (one
    // 512-thread block per SM), 64 x 4 for FP16 (two 256-thread blocks per
    // SM hide the issue-bound codec better; also fastest on the single
    // capillary and the preform)
    h->tx = 64;
    h->ty = h->half ? 4 : 8;
    const char *e = getenv("LBM_TILE");
    if (e) {
        int a = 0, b = 0;
        if (sscanf(e, "%dx%d", &a, &b) == 2) {
            h->tx = a;
            h->ty = b;
        }
    }
    const char *k = getenv("LBM_KERNEL");
    if (k && strcmp(k, "direct") == 0) h->use_tma = false;
    const char *gr = getenv("LBM_GRAPH");
    if (gr && strcmp(gr, "0") == 0) h->use_graph = false;
    // test hook of the failure path: the first step's first tile of block 0
    // waits for bytes that never arrive (the bounded wait runs out and the
    // step reports LBM_ETIMEOUT); never set in normal use
    const char *st = getenv("LBM_TEST_STALL");
    if (st) h->stall_tx = std::min(std::max(atoi(st), 0), 1 << 20);
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// One 3-D tensor map per lattice and buffer: (x, y, plane) over the
// lattice's planes of 32-bit words including the ghost band (box = the
// kernel's tile plus halo, all planes), and one over the lattice's own nodes
// (box = the tile) for the output stores; coordinates beyond read as zeros.
static bool make_maps(lbm_handle *h, std::string &why) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        why = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    const int count = h->count;
    const size_t esz = 4;
    std::vector<CUtensorMap> maps(4 * count);
    const cuuint64_t npl = h->half ? NW16 : NPOP;
    const CUtensorMapDataType pty = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    for (int b = 0; b < 2; ++b) {
        for (int l = 0; l < count; ++l) {
            const LatDesc &d = h->desc[l];
            const cuuint64_t rows = (cuuint64_t)(d.ny + 2 * GHOST);
            cuuint64_t dims[3] = {(cuuint64_t)d.pitch, rows, npl};
            cuuint64_t strides[2] = {(cuuint64_t)d.pitch * esz, (cuuint64_t)d.plane * esz};
            cuuint32_t box[3] = {(cuuint32_t)tma_box_x(h->tx),
                                 (cuuint32_t)(h->ty + 4), (cuuint32_t)npl};
            cuuint32_t es[3] = {1, 1, 1};
            void *base = (char *)h->d_pop[b] +
                         (size_t)(d.pop_off - GHOST * d.pitch - XGHOST) * esz;
            CUresult r = enc(&maps[b * count + l], pty, 3, base, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                why = "cuTensorMapEncodeTiled failed for populations, code " +
                      std::to_string((int)r);
                return false;
            }
            // output: the lattice's own nodes, logical (0, 0) at the base
            // (16-byte aligned: the ghost band is 16 columns wide)
            cuuint64_t odims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, npl};
            cuuint32_t obox[3] = {(cuuint32_t)h->tx, (cuuint32_t)h->ty, (cuuint32_t)npl};
            r = enc(&maps[(2 + b) * count + l], pty, 3,
                    (char *)h->d_pop[b] + (size_t)d.pop_off * esz, odims, strides,
                    obox, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                why = "cuTensorMapEncodeTiled failed for the output, code " +
                      std::to_string((int)r);
                return false;
            }
        }
    }
    std::vector<CUtensorMap> mmaps(count);
    for (int l = 0; l < count; ++l) {
        const LatDesc &d = h->desc[l];
        cuuint64_t dims[2] = {(cuuint64_t)d.pitch, (cuuint64_t)(d.ny + 2 * GHOST)};
        cuuint64_t strides[1] = {(cuuint64_t)d.pitch};
        cuuint32_t box[2] = {(cuuint32_t)tma_mask_box_x(h->tx), (cuuint32_t)(h->ty + 4)};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&mmaps[l], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                         h->d_mask + d.node_off - GHOST * d.pitch - XGHOST, dims,
                         strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            why = "cuTensorMapEncodeTiled failed for the mask, code " +
                  std::to_string((int)r);
            return false;
        }
    }
    if (cudaMalloc(&h->d_mask_maps, mmaps.size() * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMemcpy(h->d_mask_maps, mmaps.data(), mmaps.size() * sizeof(CUtensorMap),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        why = "tensor map upload";
        return false;
    }
    if (cudaMalloc(&h->d_maps, maps.size() * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMemcpy(h->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        why = "tensor map upload";
        return false;
    }
    return true;
}

// Tile schedule of the persistent TMA kernel, host arithmetic only.  A
// strip is a run of tiles down one tile column of a lattice (the halo rows
// each tile copies were just copied by the tile above it).  Columns taller
// than a quarter of a block's share (at least 4 tiles) are cut into strips
// of that length, so that a few tall lattices (a 2048-row preform: 32
// columns of 256 tiles) still spread over every block.  Strips go, longest
// first, to the block with the least work so far; block b then walks its
// strips top to bottom, its k-th tile at sched[b + k * grid] (lattice -1 =
// done).  Returns the slots per block.
static size_t plan_tiles(const int32_t *nx, const int32_t *ny, int count,
                         int tx, int ty, int grid, std::vector<TileRec> &sched) {
    struct Strip { int lat, col, row0, rows; };
    long long total = 0;
    for (int l = 0; l < count; ++l)
        total += (long long)((nx[l] + tx - 1) / tx) * ((ny[l] + ty - 1) / ty);
    const long long seg =
        std::max(4LL, (total + 4LL * grid - 1) / (4LL * grid));
    std::vector<Strip> strips;
    for (int l = 0; l < count; ++l) {
        const int cols = (nx[l] + tx - 1) / tx, rows = (ny[l] + ty - 1) / ty;
        for (int c = 0; c < cols; ++c)
            for (int r0 = 0; r0 < rows; r0 += (int)seg)
                strips.push_back({l, c, r0, (int)std::min<long long>(seg, rows - r0)});
    }
    std::stable_sort(strips.begin(), strips.end(),
                     [](const Strip &a, const Strip &b) { return a.rows > b.rows; });
    std::vector<std::vector<TileRec>> lists(grid);
    std::vector<long long> load(grid, 0);
    // blocks ordered by load with a simple binary heap
    std::vector<int> heap(grid);
    for (int b = 0; b < grid; ++b) heap[b] = b;
    auto less = [&](int a, int b) { return load[a] > load[b] || (load[a] == load[b] && a > b); };
    std::make_heap(heap.begin(), heap.end(), less);
    for (const Strip &st : strips) {
        std::pop_heap(heap.begin(), heap.end(), less);
        const int b = heap.back();
        for (int r = st.row0; r < st.row0 + st.rows; ++r)
            lists[b].push_back(TileRec{st.lat, st.col * tx, r * ty, 0});
        load[b] += st.rows;
        std::push_heap(heap.begin(), heap.end(), less);
    }
    size_t slots = 0;
    for (auto &v : lists) slots = std::max(slots, v.size());
    sched.assign((size_t)grid * slots, TileRec{-1, 0, 0, 0});
    for (int b = 0; b < grid; ++b)
        for (size_t k = 0; k < lists[b].size(); ++k) sched[b + k * grid] = lists[b][k];
    return slots;
}

static bool make_schedule(lbm_handle *h, std::string &why) {
    int grid = 0;
    cudaError_t e = grid_step_tma(h->tx, h->ty, h->store(), &grid);
    if (e != cudaSuccess || grid <= 0) {
        why = std::string("TMA kernel setup: ") + cudaGetErrorString(e);
        return false;
    }
    std::vector<int32_t> nx(h->count), ny(h->count);
    for (int l = 0; l < h->count; ++l) {
        nx[l] = h->desc[l].nx;
        ny[l] = h->desc[l].ny;
    }
    std::vector<TileRec> sched;
    const size_t slots = plan_tiles(nx.data(), ny.data(), h->count, h->tx, h->ty, grid, sched);
    if (cudaMalloc(&h->d_sched, std::max<size_t>(sched.size(), 1) * sizeof(TileRec)) != cudaSuccess ||
        cudaMemcpy(h->d_sched, sched.data(), sched.size() * sizeof(TileRec),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        why = "schedule upload";
        return false;
    }
    h->sched_grid = grid;
    h->sched_slots = (int)slots;
    return true;
}

// Re-tiles every lattice for another step kernel or tile shape: tile
// counts in the descriptors, the tile -> lattice table and, for the TMA
// kernel, the tensor maps and the block schedule.  Drops the captured graph.
static lbm_status retile(lbm_handle *h, bool tma, int tx, int ty) {
    for (cudaGraphExec_t &g : h->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    h->use_tma = tma;
    h->tx = tx;
    h->ty = ty;
    int tiles = 0;
    for (auto &d : h->desc) {
        d.tiles_x = (d.nx + tx - 1) / tx;
        d.tile_base = tiles;
        tiles += d.tiles_x * ((d.ny + ty - 1) / ty);
    }
    std::vector<int32_t> tile_lat(tiles);
    for (int l = 0; l < h->count; ++l) {
        const LatDesc &d = h->desc[l];
        const int nt = d.tiles_x * ((d.ny + ty - 1) / ty);
        for (int k = 0; k < nt; ++k) tile_lat[d.tile_base + k] = l;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->d_tile_lat) cudaFree(h->d_tile_lat);
    h->d_tile_lat = nullptr;
    CK(h, dalloc(&h->d_tile_lat, tiles));
    CK(h, cudaMemcpy(h->d_tile_lat, tile_lat.data(), tiles * sizeof(int32_t),
                     cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->d_desc, h->desc.data(), h->count * sizeof(LatDesc),
                     cudaMemcpyHostToDevice));
    h->ntiles = tiles;
    for (CUtensorMap **m : {&h->d_maps, &h->d_mask_maps}) {
        if (*m) cudaFree(*m);
        *m = nullptr;
    }
    if (h->d_sched) cudaFree(h->d_sched);
    h->d_sched = nullptr;
    if (tma) {
        std::string why;
        if (!make_maps(h, why) || !make_schedule(h, why))
            return fail(h, LBM_EINVAL, "tile shape not supported: " + why);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_create_batch(const lbm_geometry *g,
                                       const lbm_params *p, int32_t count,
                                       lbm_handle **out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g || !p || count < 1)
        return fail(nullptr, LBM_EINVAL, "geometry/params NULL or count < 1");
    std::string why;
    for (int l = 0; l < count; ++l) {
        const lbm_geometry &G = g[l];
        if (G.nx < 1 || G.ny < 3 || !G.solid || !G.rho_a || !G.rho_b ||
            !G.conc)
            return fail(nullptr, LBM_EINVAL,
                        "lattice " + std::to_string(l) +
                            ": need nx >= 1, ny >= 3 and all arrays");
        // 32-bit offsets inside a lattice: 22 planes of ny * pitch elements
        if ((int64_t)NPOP * (G.ny + 2 * GHOST) * ((G.nx + 2 * XGHOST + 31) / 32 * 32) >=
            ((int64_t)1 << 31))
            return fail(nullptr, LBM_EINVAL, "lattice too large");
        if (!(0 <= G.cap_x0 && G.cap_x0 < G.cap_x1 && G.cap_x1 <= G.nx))
            return fail(nullptr, LBM_EINVAL,
                        "lattice " + std::to_string(l) + ": bad section");
        if (!valid_params(p[l], why))
            return fail(nullptr, LBM_EINVAL,
                        "lattice " + std::to_string(l) + ": " + why);
        if (p[l].precision != p[0].precision)
            return fail(nullptr, LBM_EINVAL, "mixed precision in a batch");
    }
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation");
    h->count = count;
    h->half = p[0].precision != LBM_FP32;
    h->bf16 = p[0].precision == LBM_BF16;
    pick_tile(h);

    // ---- packed ragged layout ------------------------------------------
    h->desc.resize(count);
    h->col_base.resize(count);
    h->in_off_host.assign(count + 1, 0);
    int64_t pop = 0, node = 0, cols = 0, sec = 0;
    int tiles = 0;
    for (int l = 0; l < count; ++l) {
        const lbm_geometry &G = g[l];
        const lbm_params &P = p[l];
        LatDesc &d = h->desc[l];
        d.nx = G.nx;
        d.ny = G.ny;
        d.pitch = (G.nx + 2 * XGHOST + 31) / 32 * 32;
        d.tiles_x = (G.nx + h->tx - 1) / h->tx;
        d.tile_base = tiles;
        tiles += d.tiles_x * ((G.ny + h->ty - 1) / h->ty);
        d.cap_x0 = G.cap_x0;
        d.cap_x1 = G.cap_x1;
        d.inlet = P.inlet ? 1 : 0;
        // planes include GHOST rows on both sides; offsets point at row 0
        d.plane = (int64_t)(d.ny + 2 * GHOST) * d.pitch;
        d.node_off = node + GHOST * d.pitch + XGHOST;
        d.pop_off = pop + GHOST * d.pitch + XGHOST;
        d.pad64_ = 0;
        d.col_off = sec;
        node += d.plane;
        pop += (h->half ? NW16 : NPOP) * d.plane;
        h->col_base[l] = cols;
        cols += d.nx;
        sec += G.cap_x1 - G.cap_x0;
        d.tau_a = (float)P.tau_a;
        d.tau_b = (float)P.tau_b;
        d.inv_tau_a = (float)(1.0 / P.tau_a);
        d.inv_tau_b = (float)(1.0 / P.tau_b);
        d.inv_tau_d = (float)(1.0 / P.tau_d);
        d.g_coh = (float)P.g_coh;
        d.g_ads = (float)P.g_ads;
        d.k_r = (float)P.k_r;
        d.c_in = (float)P.c_in;
        d.body_x = (float)P.body_force_x;
        d.m_th = P.m_threshold;
        d.index = l;
        d.bf16 = h->bf16 ? 1 : 0;
        h->max_nodes = std::max(h->max_nodes, (size_t)G.nx * G.ny);
        h->in_off_host[l + 1] = h->in_off_host[l] + (int64_t)G.nx * G.ny;
    }
    h->ntiles = tiles;
    h->pop_elems = pop;
    h->node_elems = node;
    h->ncols = cols;
    h->nsec = sec;

    std::vector<int32_t> tile_lat(tiles), col_lat(cols);
    for (int l = 0; l < count; ++l) {
        const LatDesc &d = h->desc[l];
        const int nt = d.tiles_x * ((d.ny + h->ty - 1) / h->ty);
        for (int k = 0; k < nt; ++k) tile_lat[d.tile_base + k] = l;
        for (int x = 0; x < d.nx; ++x) col_lat[h->col_base[l] + x] = l;
    }
    // mask bytes, section-column counts and initial wall thicknesses are
    // built on the device from each lattice's solid array (k_mask_init,
    // k_col_init) below

    // ---- device allocations ----------------------------------------------
    const size_t esz = 4;  // 32-bit words in both storages
    cudaError_t e = cudaSuccess;
#define AL(ptr, n)                                                      \
    if (e == cudaSuccess) e = dalloc(&(ptr), (n));
    AL(h->d_desc, count);
    AL(h->d_tile_lat, tiles);
    AL(h->d_col_lat, cols);
    AL(h->d_col_base, count);
    AL(h->d_in_off, 2 * (count + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_pop[0], pop * esz);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_pop[1], pop * esz);
    AL(h->d_mask, node);
    AL(h->d_m, node);
    AL(h->d_col_fluid, sec);
    AL(h->d_wall0, 2 * sec);
    AL(h->d_st, count);
    AL(h->d_step, 1);
    AL(h->d_done, 1);
    AL(h->d_cols, cols);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_obs, count * sizeof(lbm_obs));
    AL(h->d_sums, 3 * count);
    AL(h->d_canon, NPOP * h->max_nodes);
    AL(h->d_dens, 3 * h->max_nodes);
    AL(h->d_dep, h->max_nodes);
    AL(h->d_err, 1);
#undef AL
    if (e != cudaSuccess) {
        std::string msg = std::string("device allocation: ") + cudaGetErrorString(e);
        free_all(h);
        delete h;
        cudaGetLastError();
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, msg);
    }
    lbm_status st = LBM_OK;
    auto bad = [&](cudaError_t ce, const char *what) {
        if (ce != cudaSuccess && st == LBM_OK) {
            g_create_err = std::string(what) + ": " + cudaGetErrorString(ce);
            st = LBM_ECUDA;
        }
    };
    bad(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking), "stream");
    h->stream = h->own;
    cudaStream_t s = h->stream;
    // Initial state of the whole batch: every lattice's inputs go into one
    // device staging area -- read in place by one gather kernel where the
    // device can address the caller's arrays (pinned or registered host
    // memory, device or managed memory), else copied by the host (one copy
    // per pageable array) -- issued on the handle's stream and landing
    // while the host builds the tensor maps and the schedule below; then
    // one launch per set-up kernel covers all lattices.
    const int64_t total = h->in_off_host.back();
    float *rho3 = nullptr;
    uint8_t *sol = nullptr;
    // prefixes over the lattices (count + 1 entries each): nodes (staging
    // offsets), rows, rows with the ghost band, section columns
    const int C1 = count + 1;
    int64_t *pre = nullptr;
    if (st == LBM_OK) {
        bad(dalloc(&rho3, 3 * (size_t)total), "alloc");
        bad(dalloc(&sol, (size_t)total), "alloc");
        bad(dalloc(&pre, 4 * (size_t)C1), "alloc");
    }
    std::vector<int64_t> pre_h(4 * C1, 0);
    for (int l = 0; l < count; ++l) {
        pre_h[l + 1] = h->in_off_host[l + 1];
        pre_h[C1 + l + 1] = pre_h[C1 + l] + h->desc[l].ny;
        pre_h[2 * C1 + l + 1] = pre_h[2 * C1 + l] + h->desc[l].ny + 2 * GHOST;
        pre_h[3 * C1 + l] = h->desc[l].col_off;
    }
    pre_h[3 * C1 + count] = h->nsec;
    h->total_rows = pre_h[C1 + count];
    if (st == LBM_OK) {
        bad(cudaMemcpyAsync(pre, pre_h.data(), pre_h.size() * 8, cudaMemcpyHostToDevice, s), "prefix");
        bad(cudaMemcpyAsync(h->d_in_off, pre_h.data(), 2 * C1 * 8, cudaMemcpyHostToDevice, s), "prefix");
    }
    InPtrs *d_ptrs = nullptr;
    if (st == LBM_OK) {
        std::vector<InPtrs> ptrs(count);
        bool any = false;
        for (int l = 0; l < count && st == LBM_OK; ++l) {
            const int64_t N = (int64_t)h->desc[l].nx * h->desc[l].ny, o = h->in_off_host[l];
            InPtrs &q = ptrs[l];
            q.rho_a = static_cast<const float *>(device_view(g[l].rho_a));
            q.rho_b = static_cast<const float *>(device_view(g[l].rho_b));
            q.conc = static_cast<const float *>(device_view(g[l].conc));
            q.solid = static_cast<const uint8_t *>(device_view(g[l].solid));
            any = any || q.rho_a || q.rho_b || q.conc || q.solid;
            // (the copy direction is inferred: pageable host memory, or
            // another device's memory)
            if (!q.rho_a)
                bad(cudaMemcpyAsync(rho3 + 3 * o, g[l].rho_a, N * 4, cudaMemcpyDefault, s), "rho_a");
            if (!q.rho_b)
                bad(cudaMemcpyAsync(rho3 + 3 * o + N, g[l].rho_b, N * 4, cudaMemcpyDefault, s), "rho_b");
            if (!q.conc)
                bad(cudaMemcpyAsync(rho3 + 3 * o + 2 * N, g[l].conc, N * 4, cudaMemcpyDefault, s), "conc");
            if (!q.solid)
                bad(cudaMemcpyAsync(sol + o, g[l].solid, N, cudaMemcpyDefault, s), "solid");
        }
        if (any && st == LBM_OK) {
            bad(dalloc(&d_ptrs, (size_t)count), "alloc");
            if (st == LBM_OK)
                bad(cudaMemcpyAsync(d_ptrs, ptrs.data(), count * sizeof(InPtrs),
                                    cudaMemcpyHostToDevice, s), "pointers");
            // at most 65535 lattices per launch (grid y)
            for (int l0 = 0; l0 < count && st == LBM_OK; l0 += 65535) {
                const unsigned ny_ = (unsigned)std::min(count - l0, 65535);
                k_gather_inputs<<<dim3(16, ny_), 256, 0, s>>>(d_ptrs, l0, h->d_in_off,
                                                              rho3, sol);
                bad(cudaGetLastError(), "gather");
            }
        }
    }
    // tables the kernels read (small synchronous copies on the legacy
    // stream, which the handle's stream does not wait for)
    bad(cudaMemcpy(h->d_desc, h->desc.data(), count * sizeof(LatDesc), cudaMemcpyHostToDevice), "desc");
    bad(cudaMemcpy(h->d_tile_lat, tile_lat.data(), tiles * sizeof(int32_t), cudaMemcpyHostToDevice), "tiles");
    bad(cudaMemcpy(h->d_col_lat, col_lat.data(), cols * sizeof(int32_t), cudaMemcpyHostToDevice), "cols");
    bad(cudaMemcpy(h->d_col_base, h->col_base.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice), "colbase");
    std::vector<LatState> st0(count);
    for (auto &x : st0) {
        memset(&x, 0, sizeof(x));
        x.closure = ~0ull;
    }
    bad(cudaMemcpy(h->d_st, st0.data(), count * sizeof(LatState), cudaMemcpyHostToDevice), "state");
    // the zeroed buffers on a stream of their own, behind nothing, so that
    // they run beside the gather; the host meanwhile builds the tensor maps
    // and the block schedule
    cudaStream_t s2 = nullptr;
    bad(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking), "stream");
    if (st == LBM_OK) {
        bad(cudaMemsetAsync(h->d_mask, 0, node, s2), "memset");
        bad(cudaMemsetAsync(h->d_pop[0], 0, pop * esz, s2), "memset");
        bad(cudaMemsetAsync(h->d_pop[1], 0, pop * esz, s2), "memset");
        bad(cudaMemsetAsync(h->d_m, 0, node * sizeof(double), s2), "memset");
        bad(cudaMemsetAsync(h->d_step, 0, sizeof(int64_t), s2), "memset");
        bad(cudaMemsetAsync(h->d_err, 0, sizeof(int), s2), "memset");
        bad(cudaMemsetAsync(h->d_done, 0, sizeof(unsigned), s2), "memset");
    }
    if (st == LBM_OK && h->use_tma) {
        std::string why;
        if (!make_maps(h, why) || !make_schedule(h, why)) {
            g_create_err = why;
            st = LBM_ECUDA;
        }
    }
    // the gather (handle's stream), the zeroing (s2) and the legacy-stream
    // copies all land before the set-up kernels
    if (st == LBM_OK) bad(cudaDeviceSynchronize(), "sync");
    if (s2) cudaStreamDestroy(s2);
    if (st == LBM_OK) {
        k_mask_init_all<<<(unsigned)pre_h[2 * C1 + count], 128, 0, s>>>(
            h->d_desc, count, pre + 2 * C1, pre, sol, h->d_mask);
        if (h->nsec > 0)
            k_col_init_all<<<(unsigned)((h->nsec + 255) / 256), 256, 0, s>>>(
                h->d_desc, count, pre + 3 * C1, pre, sol, h->d_col_fluid,
                h->d_wall0, h->d_st);
        k_init_rest_all<<<(unsigned)h->total_rows, 128, 0, s>>>(
            h->d_desc, count, pre + C1, pre, rho3, h->d_mask, h->d_pop[0], h->half);
        bad(cudaGetLastError(), "init kernels");
    }
    bad(cudaStreamSynchronize(s), "init sync");
    if (rho3) cudaFree(rho3);
    if (sol) cudaFree(sol);
    if (pre) cudaFree(pre);
    if (d_ptrs) cudaFree(d_ptrs);
    if (st != LBM_OK) {
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return LBM_OK;
}

extern "C" lbm_status lbm_create(const lbm_geometry *g, const lbm_params *p,
                                 lbm_handle **out) {
    return lbm_create_batch(g, p, 1, out);
}

extern "C" void lbm_destroy(lbm_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

extern "C" const char *lbm_last_error(const lbm_handle *h) {
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

extern "C" int64_t lbm_step_count(const lbm_handle *h) { return h ? h->steps : -1; }
extern "C" int32_t lbm_count(const lbm_handle *h) { return h ? h->count : 0; }

extern "C" lbm_status lbm_set_stream(lbm_handle *h, void *cuda_stream) {
    if (!h) return LBM_EINVAL;
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    CK(h, cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own;
    return LBM_OK;
}

static StepArgs step_args(lbm_handle *h) {
    StepArgs a;
    a.desc = h->d_desc;
    a.tile_lat = h->d_tile_lat;
    a.fin = h->d_pop[h->cur];
    a.fout = h->d_pop[h->cur ^ 1];
    a.mask = h->d_mask;
    a.m = h->d_m;
    a.col_fluid = h->d_col_fluid;
    a.st = h->d_st;
    a.step = h->d_step;
    a.done = h->d_done;
    a.stall_tx = h->stall_tx;
    a.sums = nullptr;
    return a;
}

// One launch of the step kernel reading buffer cur, writing cur ^ 1.  sum:
// the launch also adds up the lattice totals (zeroed first, on the stream)
// that lbm_observables then reads instead of the whole state.
static cudaError_t launch_one(lbm_handle *h, bool sum) {
    StepArgs a = step_args(h);
    if (sum) {
        cudaError_t e = cudaMemsetAsync(h->d_sums, 0, 3 * h->count * sizeof(double),
                                        h->stream);
        if (e != cudaSuccess) return e;
        a.sums = h->d_sums;
    }
    if (!h->use_tma)
        return launch_step_direct(a, h->ntiles, h->tx, h->ty, h->store(), h->stream);
    const int c = h->count, in = h->cur, out = h->cur ^ 1;
    return launch_step_tma(a, h->d_maps + in * c, h->d_mask_maps,
                           h->d_maps + (2 + out) * c, h->d_sched, h->sched_slots,
                           h->sched_grid, h->tx, h->ty, h->store(), h->d_err,
                           h->stream);
}

// Steps per captured graph: even, so a replay starts and ends with the
// same population buffer as input.
static const int kGraphSteps = 16;

// Captures kGraphSteps launches starting from buffer 0 into h->graph[sum];
// sum: the last one adds up the lattice totals.
static lbm_status capture_graph(lbm_handle *h, int sum) {
    const int cur0 = h->cur;
    h->cur = 0;
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
        e = launch_one(h, sum && k == kGraphSteps - 1);
        h->cur ^= 1;
    }
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    h->cur = cur0;
    CK(h, e);
    CK(h, e2);
    cudaError_t e3 = cudaGraphInstantiate(&h->graph[sum], g, 0);
    cudaGraphDestroy(g);
    CK(h, e3);
    return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_handle *h, int64_t n) {
    if (!h || n < 0) return fail(h, LBM_EINVAL, "bad handle or n < 0");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    // The last launch of the call adds up the lattice totals of the state it
    // leaves (a replay that ends the call uses the graph whose last launch
    // sums).
    // Whole groups of kGraphSteps steps replay one captured graph (the
    // step count lives on the device, so the graph needs no new arguments)
    // (a pending test stall is never captured into the graph)
    if (n > 0) h->sums_step = -1;
    while (h->use_graph && h->stall_tx == 0 &&
           n >= kGraphSteps + (h->cur ? 1 : 0)) {
        if (h->cur) {  // one plain step to get back to buffer 0
            CK(h, launch_one(h, false));
            h->cur ^= 1;
            h->steps += 1;
            n -= 1;
        }
        const int sum = n == kGraphSteps;
        if (!h->graph[sum]) {
            lbm_status st = capture_graph(h, sum);
            if (st != LBM_OK) return st;
        }
        CK(h, cudaGraphLaunch(h->graph[sum], h->stream));
        h->steps += kGraphSteps;
        n -= kGraphSteps;
        if (sum) h->sums_step = h->steps;
    }
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = launch_one(h, k == n - 1);
        if (e == cudaErrorInvalidValue && k == 0)
            return fail(h, LBM_EINVAL, "unsupported tile shape");
        CK(h, e);
        h->stall_tx = 0;  // the test stall applies to one launch
        h->cur ^= 1;
        h->steps += 1;
        if (k == n - 1) h->sums_step = h->steps;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_observables(lbm_handle *h, lbm_obs *out) {
    if (!h || !out) return fail(h, LBM_EINVAL, "NULL argument");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    // 32 columns per block, OBS_ROWS warps splitting their rows
    // the last step launch summed the stored totals: the column pass then
    // reads the mask and the nodes that turned solid, not the whole state
    const bool summed = h->sums_step == h->steps;
    const int nb = (int)((h->ncols + 31) / 32);
    launch_obs_columns(summed, h->store(), nb, (int)h->ncols, h->d_desc,
                       h->d_col_lat, h->d_col_base, h->d_pop[h->cur], h->d_mask,
                       h->d_m, h->steps, h->d_cols, h->stream);
    k_obs_reduce<<<h->count, 256, 0, h->stream>>>(
        h->d_desc, h->d_col_base, h->d_cols, h->d_wall0, h->d_st,
        summed ? h->d_sums : nullptr, h->steps, (LbmObsDev *)h->d_obs);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(out, h->d_obs, h->count * sizeof(lbm_obs),
                          cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    int kerr = 0;
    CK(h, cudaMemcpy(&kerr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (kerr) {
        h->dead = true;
        return fail(h, LBM_ETIMEOUT, "a bounded wait in the step kernel ran out");
    }
    for (int l = 0; l < h->count; ++l)
        if (out[l].nonfinite)
            return fail(h, LBM_ENAN, "non-finite density in lattice " + std::to_string(l));
    return LBM_OK;
}

extern "C" lbm_status lbm_get_solid_mask(lbm_handle *h, int32_t k,
                                         uint8_t *host, size_t n) {
    if (!h || !host || k < 0 || k >= h->count) return fail(h, LBM_EINVAL, "bad argument");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    const LatDesc &d = h->desc[k];
    if (n != (size_t)d.nx * d.ny) return fail(h, LBM_EINVAL, "size mismatch");
    // extracted on the device into the export scratch (max_nodes floats)
    const MaskBits mb(h->steps);
    uint8_t *tmp = reinterpret_cast<uint8_t *>(h->d_canon);
    k_solid_mask<<<dim3((d.nx + 127) / 128, d.ny), 128, 0, h->stream>>>(
        h->d_desc, k, h->d_mask, mb.force, tmp);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(host, tmp, n, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_get_solid_masks(lbm_handle *h, uint8_t *host,
                                          size_t n) {
    if (!h || !host) return fail(h, LBM_EINVAL, "bad argument");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    const int64_t total = h->in_off_host.back();
    if (n != (size_t)total) return fail(h, LBM_EINVAL, "size mismatch");
    // device scratch, then one copy (into pinned memory the copy runs at
    // the link's rate; the kernel writing pinned memory itself measured
    // slower, 1.07 against 0.77 ms for 105 MB)
    if (!h->d_masks) CK(h, dalloc(&h->d_masks, (size_t)total));
    const MaskBits mb(h->steps);
    k_solid_mask_all<<<(unsigned)h->total_rows, 128, 0, h->stream>>>(
        h->d_desc, h->count, h->d_in_off + h->count + 1, h->d_in_off, h->d_mask,
        mb.force, h->d_masks);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(host, h->d_masks, n, cudaMemcpyDefault, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_get_fields(lbm_handle *h, int32_t k, int32_t which,
                                     void *host, size_t bytes) {
    if (!h || !host || k < 0 || k >= h->count) return fail(h, LBM_EINVAL, "bad argument");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    const LatDesc &d = h->desc[k];
    const size_t N = (size_t)d.nx * d.ny;
    size_t need = which == LBM_FIELD_POPS ? NPOP * N * 4
                : which == LBM_FIELD_DEPOSIT ? N * 8
                : which == LBM_FIELD_DENSITY ? 3 * N * 4 : 0;
    if (need == 0) return fail(h, LBM_EINVAL, "unknown field");
    if (bytes != need) return fail(h, LBM_EINVAL, "size mismatch");
    dim3 grid((d.nx + 127) / 128, d.ny), blk(128);
    k_export<<<grid, blk, 0, h->stream>>>(
        h->d_desc, k, h->d_pop[h->cur], h->d_mask, h->d_m, h->steps, h->half, which == LBM_FIELD_POPS ? h->d_canon : nullptr,
        which == LBM_FIELD_DENSITY ? h->d_dens : nullptr,
        which == LBM_FIELD_DEPOSIT ? h->d_dep : nullptr);
    CK(h, cudaGetLastError());
    const void *src = which == LBM_FIELD_POPS ? (const void *)h->d_canon
                    : which == LBM_FIELD_DENSITY ? (const void *)h->d_dens
                    : (const void *)h->d_dep;
    CK(h, cudaMemcpyAsync(host, src, need, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

// Folds pending flips of lattice k into its ledger and aligns its mask bits.
static lbm_status settle(lbm_handle *h, int k) {
    const LatDesc &d = h->desc[k];
    dim3 grid((d.nx + 127) / 128, d.ny), blk(128);
    k_settle<<<grid, blk, 0, h->stream>>>(h->d_desc, k, h->d_pop[h->cur],
                                         h->d_mask, h->d_m, h->d_st, h->steps,
                                         h->half);
    k_mask_agree<<<grid, blk, 0, h->stream>>>(h->d_desc, k, h->d_mask, h->steps);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

extern "C" lbm_status lbm_set_fields(lbm_handle *h, int32_t k, int32_t which,
                                     const void *host, size_t bytes) {
    if (!h || !host || k < 0 || k >= h->count) return fail(h, LBM_EINVAL, "bad argument");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    const LatDesc &d = h->desc[k];
    const size_t N = (size_t)d.nx * d.ny;
    h->sums_step = -1;  // the last step's lattice totals no longer hold
    if (which == LBM_FIELD_POPS) {
        if (bytes != NPOP * N * 4) return fail(h, LBM_EINVAL, "size mismatch");
        lbm_status s = settle(h, k);
        if (s != LBM_OK) return s;
        CK(h, cudaMemcpyAsync(h->d_canon, host, bytes, cudaMemcpyHostToDevice, h->stream));
        dim3 grid((d.nx + 127) / 128, d.ny), blk(128);
        const MaskBits mb(h->steps);
        k_unstream<<<grid, blk, 0, h->stream>>>(h->d_desc, k, h->d_canon, h->d_mask,
                                               mb.force, h->d_pop[h->cur],
                                               h->half);
        CK(h, cudaGetLastError());
        CK(h, cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    if (which == LBM_FIELD_DEPOSIT) {
        if (bytes != N * 8) return fail(h, LBM_EINVAL, "size mismatch");
        lbm_status s = settle(h, k);
        if (s != LBM_OK) return s;
        const size_t rows_n = (size_t)d.ny * d.pitch;
        std::vector<uint8_t> raw(rows_n);
        CK(h, cudaMemcpyAsync(raw.data(), h->d_mask + d.node_off, rows_n,
                              cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        std::vector<double> m(rows_n, 0.0);
        const double *src = static_cast<const double *>(host);
        for (int y = 0; y < d.ny; ++y)
            for (int x = 0; x < d.nx; ++x)
                if (!(raw[(size_t)y * d.pitch + x] & 7)) {
                    const double v = src[(size_t)y * d.nx + x];
                    // a fluid node at or above the threshold would have
                    // turned solid when its deposit crossed it
                    if (!(v >= 0.0 && v < d.m_th))
                        return fail(h, LBM_EINVAL,
                                    "deposit outside [0, m_threshold) at a fluid node");
                    m[(size_t)y * d.pitch + x] = v;
                }
        CK(h, cudaMemcpyAsync(h->d_m + d.node_off, m.data(), rows_n * 8,
                              cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return LBM_OK;
    }
    return fail(h, LBM_EINVAL, "field cannot be set");
}

// ---- checkpoints -----------------------------------------------------------

static const char kMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '5'};

struct CkptHeader {
    char magic[8];
    int32_t count, half;  // half: the storage, 0 FP32, 1 FP16, 2 BF16
    int64_t pop_elems, node_elems, nsec, steps;
    int32_t cur, pad;
};

extern "C" lbm_status lbm_save(lbm_handle *h, const char *path) {
    if (!h || !path) return fail(h, LBM_EINVAL, "NULL argument");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    CK(h, cudaStreamSynchronize(h->stream));
    const size_t esz = 4;
    CkptHeader hd;
    memcpy(hd.magic, kMagic, 8);
    hd.count = h->count;
    hd.half = h->store();
    hd.pop_elems = h->pop_elems;
    hd.node_elems = h->node_elems;
    hd.nsec = h->nsec;
    hd.steps = h->steps;
    hd.cur = 0;
    hd.pad = 0;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(h, LBM_EIO, std::string("cannot open ") + path);
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && fwrite(h->desc.data(), sizeof(LatDesc), h->count, f) == (size_t)h->count;
    auto dump = [&](const void *dptr, size_t bytes) {
        if (!ok) return;
        std::vector<uint8_t> buf(std::min<size_t>(bytes, (size_t)1 << 28));
        size_t done = 0;
        while (ok && done < bytes) {
            const size_t n = std::min(buf.size(), bytes - done);
            if (cudaMemcpy(buf.data(), (const uint8_t *)dptr + done, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
                ok = false;
                return;
            }
            ok = fwrite(buf.data(), 1, n, f) == n;
            done += n;
        }
    };
    dump(h->d_pop[h->cur], h->pop_elems * esz);
    dump(h->d_mask, h->node_elems);
    dump(h->d_m, h->node_elems * 8);
    dump(h->d_col_fluid, h->nsec * 4);
    dump(h->d_st, h->count * sizeof(LatState));
    dump(h->d_step, 8);
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(h, LBM_EIO, std::string("write failed: ") + path);
    return LBM_OK;
}

extern "C" lbm_status lbm_load(lbm_handle *h, const char *path) {
    if (!h || !path) return fail(h, LBM_EINVAL, "NULL argument");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    CK(h, cudaStreamSynchronize(h->stream));
    FILE *f = fopen(path, "rb");
    if (!f) return fail(h, LBM_EIO, std::string("cannot open ") + path);
    CkptHeader hd;
    bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, kMagic, 8) == 0;
    ok = ok && hd.count == h->count && hd.half == h->store() &&
         hd.pop_elems == h->pop_elems && hd.node_elems == h->node_elems &&
         hd.nsec == h->nsec;
    std::vector<LatDesc> dsc(h->count);
    ok = ok && fread(dsc.data(), sizeof(LatDesc), h->count, f) == (size_t)h->count;
    if (ok) {
        for (int l = 0; l < h->count; ++l)
            if (memcmp(&dsc[l], &h->desc[l], sizeof(LatDesc)) != 0) ok = false;
    }
    if (!ok) {
        fclose(f);
        return fail(h, LBM_EINVAL, "checkpoint does not match this handle");
    }
    const size_t esz = 4;
    auto slurp = [&](void *dptr, size_t bytes) {
        if (!ok) return;
        std::vector<uint8_t> buf(std::min<size_t>(bytes, (size_t)1 << 28));
        size_t done = 0;
        while (ok && done < bytes) {
            const size_t n = std::min(buf.size(), bytes - done);
            ok = fread(buf.data(), 1, n, f) == n;
            if (ok && cudaMemcpy((uint8_t *)dptr + done, buf.data(), n, cudaMemcpyHostToDevice) != cudaSuccess)
                ok = false;
            done += n;
        }
    };
    h->cur = 0;
    slurp(h->d_pop[0], h->pop_elems * esz);
    slurp(h->d_mask, h->node_elems);
    slurp(h->d_m, h->node_elems * 8);
    slurp(h->d_col_fluid, h->nsec * 4);
    slurp(h->d_st, h->count * sizeof(LatState));
    slurp(h->d_step, 8);
    fclose(f);
    if (!ok) return fail(h, LBM_EIO, std::string("read failed: ") + path);
    h->steps = hd.steps;
    h->sums_step = -1;
    return LBM_OK;
}

extern "C" lbm_status lbm_plan_tiles(const int32_t *nx, const int32_t *ny,
                                     int32_t count, int32_t tx, int32_t ty,
                                     int32_t grid, int32_t *out, int64_t cap,
                                     int32_t *slots) {
    if (!nx || !ny || !slots || count < 1 || tx < 1 || ty < 1 || grid < 1)
        return fail(nullptr, LBM_EINVAL, "plan_tiles: NULL array, count, tile or grid < 1");
    for (int l = 0; l < count; ++l)
        if (nx[l] < 1 || ny[l] < 1)
            return fail(nullptr, LBM_EINVAL, "plan_tiles: lattice size < 1");
    std::vector<TileRec> sched;
    const size_t n = plan_tiles(nx, ny, count, tx, ty, grid, sched);
    *slots = (int32_t)n;
    if (!out) return LBM_OK;
    if ((int64_t)sched.size() * 3 > cap)
        return fail(nullptr, LBM_EINVAL, "plan_tiles: output holds fewer than 3 * grid * slots values");
    for (size_t k = 0; k < sched.size(); ++k) {
        out[3 * k] = sched[k].lat;
        out[3 * k + 1] = sched[k].lat >= 0 ? sched[k].x0 : 0;
        out[3 * k + 2] = sched[k].lat >= 0 ? sched[k].y0 : 0;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_fit_reff(const double *t, const double *z,
                                   int32_t n, double gamma, double mu,
                                   double length, double cos_theta0,
                                   double *r_eff) {
    if (!t || !z || !r_eff || n < 2 || !(gamma > 0) || !(cos_theta0 != 0))
        return LBM_EINVAL;
    double st = 0, sz = 0;
    for (int i = 0; i < n; ++i) { st += t[i]; sz += z[i]; }
    const double mt = st / n, mz = sz / n;
    double num = 0, den = 0;
    for (int i = 0; i < n; ++i) {
        num += (t[i] - mt) * (z[i] - mz);
        den += (t[i] - mt) * (t[i] - mt);
    }
    if (!(den > 0)) return LBM_EINVAL;
    const double v = num / den;
    *r_eff = 3.0 * mu * length * v / (gamma * cos_theta0);
    return LBM_OK;
}

// ---- autotuner ---------------------------------------------------------------

extern "C" lbm_status lbm_get_tuning(const lbm_handle *h, lbm_tuning *out) {
    if (!h || !out) return LBM_EINVAL;
    out->kernel = h->use_tma ? 1 : 0;
    out->tx = h->tx;
    out->ty = h->ty;
    out->ms_per_step = 0.0;
    return LBM_OK;
}

extern "C" lbm_status lbm_autotune(lbm_handle *h, int32_t steps,
                                   lbm_tuning *out) {
    if (!h || steps < 1) return fail(h, LBM_EINVAL, "bad handle or steps < 1");
    if (h->dead) return fail(h, LBM_ECUDA, "handle is dead: " + h->err);
    CK(h, cudaStreamSynchronize(h->stream));
    // snapshot of everything a step changes
    const size_t esz = 4;
    struct Piece { void *dev; size_t bytes; };
    const int cur0 = h->cur;
    const int64_t steps0 = h->steps;
    std::vector<Piece> parts = {
        {h->d_pop[cur0], (size_t)h->pop_elems * esz},
        {h->d_mask, (size_t)h->node_elems},
        {h->d_m, (size_t)h->node_elems * 8},
        {h->d_col_fluid, (size_t)h->nsec * 4},
        {h->d_st, (size_t)h->count * sizeof(LatState)},
        {h->d_step, 8}};
    size_t total = 0;
    for (auto &p : parts) total += (p.bytes + 255) / 256 * 256;
    char *snap = nullptr;
    if (cudaMalloc(&snap, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LBM_ENOMEM, "autotune: no room for a state copy");
    }
    auto copy_all = [&](bool save) -> cudaError_t {
        size_t off = 0;
        for (auto &p : parts) {
            cudaError_t e = save ? cudaMemcpyAsync(snap + off, p.dev, p.bytes,
                                                   cudaMemcpyDeviceToDevice, h->stream)
                                 : cudaMemcpyAsync(p.dev, snap + off, p.bytes,
                                                   cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return e;
            off += (p.bytes + 255) / 256 * 256;
        }
        return cudaStreamSynchronize(h->stream);
    };
    struct Cand { bool tma; int tx, ty; };
    const Cand cands[] = {{true, 32, 16}, {true, 32, 8},  {true, 64, 4},
                          {true, 64, 8},  {true, 32, 4},  {true, 128, 4},
                          {false, 32, 8}, {false, 32, 4}, {false, 64, 4},
                          {false, 128, 4}};
    const Cand orig = {h->use_tma, h->tx, h->ty};
    Cand best = orig;
    double best_ms = 1e300;
    lbm_status st = LBM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = copy_all(true);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    for (const Cand &c : cands) {
        if (ce != cudaSuccess || st != LBM_OK) break;
        if (retile(h, c.tma, c.tx, c.ty) != LBM_OK) {
            st = LBM_OK;  // shape not available on this device: skip it
            h->err.clear();
            continue;
        }
        st = lbm_step(h, kGraphSteps + 2);  // warm-up, graph capture
        if (st != LBM_OK) break;
        const int n = (steps + kGraphSteps - 1) / kGraphSteps * kGraphSteps;
        ce = cudaEventRecord(e0, h->stream);
        if (ce == cudaSuccess) st = lbm_step(h, n);
        if (ce == cudaSuccess && st == LBM_OK) ce = cudaEventRecord(e1, h->stream);
        if (ce == cudaSuccess && st == LBM_OK) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess && st == LBM_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce == cudaSuccess && st == LBM_OK && ms / n < best_ms) {
            best_ms = ms / n;
            best = c;
        }
        // back to the saved state (its lattice totals are not kept)
        if (ce == cudaSuccess) ce = copy_all(false);
        h->cur = cur0;
        h->steps = steps0;
        h->sums_step = -1;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(snap);
    if (st != LBM_OK) return st;
    CK(h, ce);
    lbm_status r = retile(h, best.tma, best.tx, best.ty);
    if (r != LBM_OK) return r;
    if (out) {
        out->kernel = best.tma ? 1 : 0;
        out->tx = best.tx;
        out->ty = best.ty;
        out->ms_per_step = best_ms;
    }
    return LBM_OK;
}
