// lbm_step_tma.cu -- the fused reactive step with TMA-staged tiles
// (sm_103a).  Same per-node work as the direct kernel in lbm_step.cu; what
// differs is how the populations reach the SM:
//
//   * the kernel is persistent: a grid of (SM count x resident blocks)
//     walks the tiles of every lattice of the batch;
//   * for each tile of TX x TY nodes, one thread issues a single 3-D bulk
//     tensor copy (cp.async.bulk.tensor) of all 22 population planes over
//     the tile plus a halo of 2 rows and 4 (FP32) or 8 (FP16) columns --
//     the x start stays 16-byte aligned -- into shared memory, completing
//     on an mbarrier; FP16 storage adds a second copy of the 3 moment
//     planes;
//   * two stages: the copy of the next tile is in flight while the current
//     one is computed;
//   * all pulls -- the tile's own nodes and the one-node density ring the
//     cohesion stencil needs -- then read shared memory at fixed offsets;
//   * halo cells outside the lattice (the copy fills them with zeros) are
//     patched with their periodic images by plain loads, only on tiles that
//     touch a lattice edge;
//   * every wait on an mbarrier is bounded; on time-out the kernel records
//     an error, lets its copies in flight land and returns.
#include <cuda.h>

#include "lbm_node.cuh"

namespace lbmk {

// ---- PTX wrappers ----------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; gives up after
// about two seconds (or 2^26 polls) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar,
                                                  unsigned parity) {
    const long long t0 = clock64();
    for (unsigned it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > 4000000000LL) break;
    }
    return false;
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map,
                                            int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::"
        "bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2),
        "r"(smem_u32(bar))
        : "memory");
}

// ---- tile geometry -----------------------------------------------------------

template <class S, int TX_, int TY_>
struct TmaTile {
    using T = typename S::T;
    static constexpr int TX = TX_, TY = TY_;
    static constexpr int NT = TX * TY;
    static constexpr int XO = S::kHalf ? 8 : 4;  // halo columns copied
    static constexpr int BX = TX + 2 * XO;        // box width
    static constexpr int BY = TY + 4;             // box height (halo 2)
    static constexpr int PL = BX * BY;            // elements per plane
    static constexpr int POP_BYTES = NPOP * PL * (int)sizeof(T);
    static constexpr int MOM_BYTES = S::kHalf ? NMOM * PL * 2 : 0;
    static constexpr int STAGE = ((POP_BYTES + MOM_BYTES) + 127) / 128 * 128;
    static constexpr int HX = TX + 4, HY = TY + 4;  // mask halo, radius 2
    static constexpr int RX = TX + 2, RY = TY + 2;  // density frame
    static constexpr int NRING = 2 * RX + 2 * TY;
    static constexpr int MASK_BYTES = (HX * HY + 127) / 128 * 128;
    static constexpr int RHO_BYTES = (2 * RX * RY * 4 + 127) / 128 * 128;
    static constexpr int SMEM = 2 * STAGE + MASK_BYTES + RHO_BYTES + 128;
    static_assert(POP_BYTES % 128 == 0, "stage alignment");
    static_assert((BX * (int)sizeof(T)) % 16 == 0, "TMA box row");
};

// The 9 populations of component `comp` pulled into the node at stage cell
// (yy, xx), from shared memory.
template <class S, class TT>
__device__ __forceinline__ void spull9(const typename S::T *tile,
                                       const __half *mom, int comp, int yy,
                                       int xx, unsigned bb, float f[Q]) {
    const int c = yy * TT::BX + xx;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool b = (bb >> i) & 1u;
        const int cell = b ? c : c - cy(i) * TT::BX - cx(i);
        const int q = comp * Q + (b ? opp(i) : i);
        if constexpr (!S::kHalf) {
            f[i] = tile[q * TT::PL + cell];
        } else {
            f[i] = wq(i) * (__half2float(mom[comp * TT::PL + cell]) +
                            __half2float(tile[q * TT::PL + cell]));
        }
    }
}

template <class S, class TT>
__device__ __forceinline__ void spull4(const typename S::T *tile,
                                       const __half *mom, int yy, int xx,
                                       unsigned bb4, float g[QS]) {
    const int c = yy * TT::BX + xx;
#pragma unroll
    for (int k = 0; k < QS; ++k) {
        const bool b = (bb4 >> k) & 1u;
        const int cell = b ? c : c - sy(k) * TT::BX - sx(k);
        const int q = 2 * Q + (b ? sopp(k) : k);
        if constexpr (!S::kHalf) {
            g[k] = tile[q * TT::PL + cell];
        } else {
            g[k] = 0.25f * (__half2float(mom[2 * TT::PL + cell]) +
                            __half2float(tile[q * TT::PL + cell]));
        }
    }
}

template <class S, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
    k_step_tma(StepArgs a, const CUtensorMap *__restrict__ pop_maps,
               const CUtensorMap *__restrict__ mom_maps, int ntiles,
               int *__restrict__ err) {
    using TT = TmaTile<S, TX, TY>;
    using T = typename S::T;
    extern __shared__ __align__(128) unsigned char smem[];
    auto stage_pop = [&](int s) { return reinterpret_cast<T *>(smem + s * TT::STAGE); };
    auto stage_mom = [&](int s) {
        return reinterpret_cast<__half *>(smem + s * TT::STAGE + TT::POP_BYTES);
    };
    uint8_t(*smask)[TT::HX] =
        reinterpret_cast<uint8_t(*)[TT::HX]>(smem + 2 * TT::STAGE);
    float(*srho)[TT::RY][TT::RX] = reinterpret_cast<float(*)[TT::RY][TT::RX]>(
        smem + 2 * TT::STAGE + TT::MASK_BYTES);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * TT::STAGE +
                                                 TT::MASK_BYTES + TT::RHO_BYTES);
    long long *s_t = reinterpret_cast<long long *>(bar + 2);

    const int tid = threadIdx.x;
    const T *__restrict__ fin = static_cast<const T *>(a.fin);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        *s_t = *(volatile long long *)a.step;
    }
    __syncthreads();
    const long long t = *s_t;
    const MaskBits mb(t);

    auto issue = [&](int tile, int s) {
        const int l = a.tile_lat[tile];
        const LatDesc &dd = a.desc[l];
        const int local = tile - dd.tile_base;
        const int x0 = (local % dd.tiles_x) * TX - TT::XO;
        const int y0 = (local / dd.tiles_x) * TY - 2;
        fence_proxy_async();
        mbar_expect_tx(&bar[s], TT::POP_BYTES + TT::MOM_BYTES);
        tma_load_3d(stage_pop(s), &pop_maps[l], x0, y0, 0, &bar[s]);
        if constexpr (S::kHalf)
            tma_load_3d(stage_mom(s), &mom_maps[l], x0, y0, 0, &bar[s]);
    };

    int tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) issue(tile, 0);
    unsigned parity = 0u;  // bit s: phase parity of stage s
    bool failed = false;
    for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
        const int s = k & 1;
        const int next = tile + gridDim.x;
        if (tid == 0 && next < ntiles) issue(next, s ^ 1);

        const int l = a.tile_lat[tile];
        const LatDesc d = a.desc[l];
        const int nx = d.nx, ny = d.ny;
        const int local = tile - d.tile_base;
        const int tx0 = (local % d.tiles_x) * TX;
        const int ty0 = (local / d.tiles_x) * TY;
        const bool edge = tx0 < 2 || ty0 < 2 || tx0 + TX + 2 > nx ||
                          ty0 + TY + 2 > ny;
        uint8_t *__restrict__ mask = a.mask + d.node_off;

        // mask halo (plain loads; overlaps the copy in flight)
        for (int e = tid; e < TT::HY * TT::HX; e += TT::NT) {
            const int hy = e / TT::HX, hx = e - hy * TT::HX;
            int gy = ty0 - 2 + hy, gx = tx0 - 2 + hx;
            if (edge) {
                gy = wrapg(gy, ny);
                gx = wrapg(gx, nx);
            }
            smask[hy][hx] = mask[(int64_t)gy * d.pitch + gx];
        }

        // wait for this tile's copy (bounded; the decision is block-uniform)
        const bool ok = mbar_wait_bounded(&bar[s], (parity >> s) & 1u);
        parity ^= 1u << s;
        if (__syncthreads_or(!ok)) {
            failed = true;
            if (tid == 0) {
                atomicOr(err, 1);
                if (next < ntiles) mbar_wait_bounded(&bar[s ^ 1], (parity >> (s ^ 1)) & 1u);
            }
            break;
        }
        T *tp = stage_pop(s);
        __half *tm = stage_mom(s);

        // periodic images of halo cells outside the lattice
        if (edge) {
            const T *__restrict__ src = fin + d.pop_off;
            constexpr int NPL = NPOP + (S::kHalf ? NMOM : 0);
            constexpr int CW = TX + 4;  // columns needed: x0 - 2 .. x0 + TX + 1
            for (int e = tid; e < TT::BY * CW * NPL; e += TT::NT) {
                const int q = e / (TT::BY * CW);
                const int r = e - q * (TT::BY * CW);
                const int yy = r / CW;
                const int xx = r - yy * CW + TT::XO - 2;
                const int gy = ty0 - 2 + yy, gx = tx0 - TT::XO + xx;
                if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) continue;
                const int64_t g = (int64_t)wrapg(gy, ny) * d.pitch + wrapg(gx, nx);
                if (q < NPOP) {
                    tp[q * TT::PL + yy * TT::BX + xx] = src[q * d.plane + g];
                } else if constexpr (S::kHalf) {
                    tm[(q - NPOP) * TT::PL + yy * TT::BX + xx] =
                        a.min_[d.mom_off + (q - NPOP) * d.plane + g];
                }
            }
        }
        __syncthreads();

        // own node: pull and density
        const int lx = tid % TX, ly = tid / TX;
        const int x = tx0 + lx, y = ty0 + ly;
        const bool active = (x < nx) && (y < ny);
        const int yy = ly + 2, xx = lx + TT::XO;
        const int hy = ly + 2, hx = lx + 2;
        const uint8_t s_own = smask[hy][hx];
        const bool own_pull_fluid = !(s_own & mb.pull);
        float fA[Q], fB[Q];
        {
            float ra = 0.f, rb = 0.f;
            if (own_pull_fluid) {
                unsigned bb = 0;
#pragma unroll
                for (int i = 1; i < Q; ++i)
                    if (smask[hy - cy(i)][hx - cx(i)] & mb.pull) bb |= 1u << i;
                spull9<S, TT>(tp, tm, 0, yy, xx, bb, fA);
                spull9<S, TT>(tp, tm, 1, yy, xx, bb, fB);
#pragma unroll
                for (int i = 0; i < Q; ++i) { ra += fA[i]; rb += fB[i]; }
            }
            const bool force_solid = s_own & mb.force;
            srho[0][ly + 1][lx + 1] = force_solid ? 0.f : ra;
            srho[1][ly + 1][lx + 1] = force_solid ? 0.f : rb;
        }
        // ring of the density frame
        for (int r = tid; r < TT::NRING; r += TT::NT) {
            int ry, rx;
            if (r < TT::RX) { ry = 0; rx = r; }
            else if (r < 2 * TT::RX) { ry = TT::RY - 1; rx = r - TT::RX; }
            else if (r < 2 * TT::RX + TY) { ry = 1 + r - 2 * TT::RX; rx = 0; }
            else { ry = 1 + r - 2 * TT::RX - TY; rx = TT::RX - 1; }
            const uint8_t sr = smask[ry + 1][rx + 1];
            float ra = 0.f, rb = 0.f;
            if (!(sr & mb.force)) {
                unsigned bb = 0;
#pragma unroll
                for (int i = 1; i < Q; ++i)
                    if (smask[ry + 1 - cy(i)][rx + 1 - cx(i)] & mb.pull) bb |= 1u << i;
                float f[Q];
                spull9<S, TT>(tp, tm, 0, ry + 1, rx + TT::XO - 1, bb, f);
#pragma unroll
                for (int i = 0; i < Q; ++i) ra += f[i];
                spull9<S, TT>(tp, tm, 1, ry + 1, rx + TT::XO - 1, bb, f);
#pragma unroll
                for (int i = 0; i < Q; ++i) rb += f[i];
            }
            srho[0][ry][rx] = ra;
            srho[1][ry][rx] = rb;
        }
        __syncthreads();

        if (active) {
            const int64_t own = (int64_t)y * d.pitch + x;
            unsigned bb4 = 0;
#pragma unroll
            for (int k4 = 0; k4 < QS; ++k4)
                if (smask[hy - sy(k4)][hx - sx(k4)] & mb.pull) bb4 |= 1u << k4;
            if (s_own & mb.force) {
                const uint8_t nb = s_own | mb.next;
                if (own_pull_fluid) {
                    float g[QS];
                    spull4<S, TT>(tp, tm, yy, xx, bb4, g);
                    retire_node(a, d, l, own, fA, fB, g);
                }
                if (nb != s_own) mask[own] = nb;
            } else {
                float g[QS];
                spull4<S, TT>(tp, tm, yy, xx, bb4, g);
                const bool flagged = fluid_update<S>(
                    a, d, l, t, x, own, fA, fB, g,
                    [&](int c, int i) { return srho[c][ly + 1 + cy(i)][lx + 1 + cx(i)]; },
                    [&](int i) { return (smask[hy + cy(i)][hx + cx(i)] & mb.force) != 0; },
                    [&](int k4) { return (smask[hy + sy(k4)][hx + sx(k4)] & mb.force) != 0; });
                if (flagged) mask[own] = s_own | mb.next;
            }
        }
        // stage s, the mask halo and the density frame are reused next
        __syncthreads();
    }
    (void)failed;
    finish_launch(a, t);
}

// ---- host side ---------------------------------------------------------------

template <class S, int TX, int TY>
static cudaError_t launch_tma_t(const StepArgs &a, const CUtensorMap *pop_maps,
                                const CUtensorMap *mom_maps, int ntiles,
                                int *err, cudaStream_t s) {
    using TT = TmaTile<S, TX, TY>;
    static int grid = 0;
    if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(
            k_step_tma<S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            TT::SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per, k_step_tma<S, TX, TY>, TX * TY, TT::SMEM);
        if (e != cudaSuccess) return e;
        grid = sms * (per > 0 ? per : 1);
    }
    const int g = ntiles < grid ? ntiles : grid;
    k_step_tma<S, TX, TY><<<g, TX * TY, TT::SMEM, s>>>(a, pop_maps, mom_maps,
                                                       ntiles, err);
    return cudaGetLastError();
}

cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap *pop_maps,
                            const CUtensorMap *mom_maps, int ntiles, int tx,
                            int ty, bool half, int *err, cudaStream_t s) {
#define LBM_TMA_CASE(X, Y)                                                   \
    if (tx == X && ty == Y)                                                  \
        return half ? launch_tma_t<Store16, X, Y>(a, pop_maps, mom_maps,     \
                                                  ntiles, err, s)            \
                    : launch_tma_t<Store32, X, Y>(a, pop_maps, mom_maps,     \
                                                  ntiles, err, s);
    LBM_TMA_CASE(32, 8)
    LBM_TMA_CASE(32, 4)
    LBM_TMA_CASE(64, 4)
    LBM_TMA_CASE(32, 16)
    LBM_TMA_CASE(64, 8)
#undef LBM_TMA_CASE
    return cudaErrorInvalidValue;
}

// Tensor map geometry must match TmaTile: box (TX + 2 XO) x (TY + 4) x planes.
int tma_box_x(int tx, bool half) { return tx + 2 * (half ? 8 : 4); }

}  // namespace lbmk
