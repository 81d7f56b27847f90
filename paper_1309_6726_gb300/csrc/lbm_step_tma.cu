// lbm_step_tma.cu -- the fused reactive step with TMA-staged tiles
// (sm_103a).  Same per-node work as the direct kernel in lbm_step.cu; what
// differs is how the populations reach the SM:
//
//   * the kernel is persistent: a grid of (SM count x resident blocks)
//     walks the tiles of every lattice of the batch;
//   * for each tile of TX x TY nodes, one thread issues a 3-D bulk tensor
//     copy (cp.async.bulk.tensor) of the population planes (32-bit words:
//     22 FP32 values, or the 15 words of FP16 storage) over the tile plus
//     a halo of 2 rows and 4 columns -- the x start stays 16-byte aligned
//     -- into shared memory, completing on an mbarrier; the mask box and
//     the lattice descriptor come with it;
//   * two stages: the copy of the next tile is in flight while the current
//     one is computed;
//   * all pulls -- the tile's own nodes and the one-node density ring the
//     cohesion stencil needs -- then read shared memory at fixed offsets;
//   * the tile's post-collision values go to a shared output tile that one
//     bulk tensor store per tile copies out;
//   * the lattice planes carry a two-node periodic ghost band (rows and
//     columns), so every copy reads valid neighbours and nothing needs
//     patching;
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

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map,
                                            int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::"
        "bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1),
        "r"(smem_u32(bar))
        : "memory");
}

// Bulk tensor store of a shared-memory box to global memory (elements
// outside the tensor are skipped), committed as one bulk group.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map,
                                             const void *src, int c0, int c1,
                                             int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group "
        "[%0, {%1, %2, %3}], [%4];" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
        : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// The shared memory of every committed store has been read.
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Every committed store has completed.
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src,
                                          unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- tile geometry -----------------------------------------------------------

template <class S, int TX_, int TY_>
struct TmaTile {
    using T = typename S::T;  // 32-bit words: FP32 values or 16-bit pairs
    using Fmt = typename S::Fmt;  // 16-bit format (16-bit storage)
    static constexpr int TX = TX_, TY = TY_;
    static constexpr int NT = TX * TY;
    static constexpr int NW = NT / 32;            // warps
    static constexpr int XO = 4;                  // halo columns copied (16 B)
    static constexpr int BX = TX + 2 * XO;        // box width
    static constexpr int BY = TY + 4;             // box height (halo 2)
    static constexpr int PL = BX * BY;            // words per plane
    static constexpr int MXO = 16;                // mask box: 16-byte aligned
    static constexpr int MBX = TX + 2 * MXO;
    // population planes of a stage: 22 FP32, or the 15 words of FP16 storage
    static constexpr int NPL = S::kPlanes;
    static constexpr int POP_BYTES = NPL * PL * 4;
    static constexpr int MASK_BYTES = (MBX * BY + 127) / 128 * 128;
    static constexpr int STAGE = ((POP_BYTES + 127) / 128 * 128) + MASK_BYTES;
    static constexpr int MASK_OFF = STAGE - MASK_BYTES;  // within a stage
    static constexpr int TX_BYTES = POP_BYTES + MBX * BY + 128;
    static constexpr int RX = TX + 2, RY = TY + 2;  // density frame
    static constexpr int NRING = 2 * RX + 2 * TY;
    // FP32: two planes rho_A, rho_B; FP16: one plane of {rho_A, rho_B}
    static constexpr int RHO_BYTES = 2 * RX * RY * 4;
    static constexpr int RHO_AL = (RHO_BYTES + 127) / 128 * 128;
    // Two stages: the copy of the next tile lands while this one is
    // computed (a third stage measured no faster).  One descriptor slot
    // more than stages: the current tile's stays readable while the next
    // copies land.
    static constexpr int NS = 2;
    static constexpr int NSL = NS + 1;
    static constexpr int DESC_OFF = NS * STAGE;                // NSL x 128
    static constexpr int RHO_OFF = DESC_OFF + NSL * 128;       // 2 frames
    // The tile's post-collision output, [NPL][TY][TX] words, written by
    // bulk tensor stores (FP32 storage: one output tile where it fits, two
    // block barriers per tile).  FP16 storage takes one block barrier per
    // tile (ONE_BAR): tiles of up to 256 nodes store their nodes directly
    // (coalesced 32-bit stores) and run two blocks per SM (128 registers;
    // the budget of three, 80 registers, spilled and measured 10 % slower
    // on the batched sweep at 64 x 4, whose stages leave room for two
    // blocks only); larger tiles keep two output tiles, so that the store
    // of one is issued while the next is written.
    static constexpr int OUT_BYTES = (NPL * NT * 4 + 127) / 128 * 128;
    static constexpr int OUT_OFF = RHO_OFF + 2 * RHO_AL;
    static constexpr bool ONE_BAR = S::kHalf;
    static constexpr int NOUT =
        S::kHalf ? (NT <= 256 ? 0 : (OUT_OFF + 2 * OUT_BYTES + 128 <= 232448 ? 2 : 0))
                 : (OUT_OFF + OUT_BYTES + 128 <= 232448 ? 1 : 0);
    static constexpr bool TS = NOUT > 0;
    // blocks per SM the register budget is set for
    static constexpr int MINB = S::kHalf && NT <= 256 ? 2 : 1;
    static constexpr int BAR_OFF = OUT_OFF + NOUT * OUT_BYTES;
    static constexpr int SMEM = BAR_OFF + 128;
    static_assert(SMEM <= 232448, "shared memory per block");
    static_assert((TX * 4) % 16 == 0, "store box row");
    static_assert(POP_BYTES % 16 == 0, "stage alignment");
    static_assert((BX * 4) % 16 == 0, "TMA box row");
    // ring cells per warp: whole warps take the ring (5 of 8 at 64 x 4),
    // since a warp costs the same issue slots with 10 lanes active as with
    // 32 (spreading it thinly over every warp measured 4 % slower for FP16)
    static constexpr int RW = 32;
    static_assert(NRING <= NT && RW <= 32, "ring spread");
    static_assert(TX % 32 == 0, "a warp covers 32 columns of one row");
};

// The 9 populations of component `comp` pulled into the node at stage cell
// `c`, from shared memory (bb: bounce-back bits), FP32 storage.  BB = false:
// no source is solid, every address is the node's cell plus a constant.
template <class TT, bool BB>
__device__ __forceinline__ void spull9(const float *tile, int comp, int c,
                                       unsigned bb, float f[Q]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const bool b = BB && ((bb >> i) & 1u);
        const int cell = b ? c : c - cy(i) * TT::BX - cx(i);
        const int qi = b ? opp(i) : i;
        f[i] = tile[(comp * Q + qi) * TT::PL + cell];
    }
}

template <class TT, bool BB>
__device__ __forceinline__ void spull4(const float *tile, int c, unsigned bb4,
                                       float g[QS]) {
#pragma unroll
    for (int k = 0; k < QS; ++k) {
        const bool b = BB && ((bb4 >> k) & 1u);
        const int cell = b ? c : c - sy(k) * TT::BX - sx(k);
        g[k] = tile[(2 * Q + (b ? sopp(k) : k)) * TT::PL + cell];
    }
}

// FP16 storage: the scaled {A, B} populations pulled into the node at
// stage cell c -- per direction one packed deviation word, the source's two
// FP32 references and its one or two linear-reference words; the rest
// populations are the node's own references.
template <class TT, bool BB>
__device__ __forceinline__ void spull16ab(const uint32_t *tile, int c,
                                          unsigned bb, float2 f[Q]) {
    const float *ref = reinterpret_cast<const float *>(tile) + W16_REF * TT::PL;
    f[0] = make_float2(ref[c], ref[TT::PL + c]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const bool b = BB && ((bb >> i) & 1u);
        const int cell = b ? c : c - cy(i) * TT::BX - cx(i);
        const int qi = b ? opp(i) : i;
        const uint32_t wx = cx(i) != 0 ? tile[W16_VEL * TT::PL + cell] : 0u;
        const uint32_t wy = cy(i) != 0 ? tile[(W16_VEL + 1) * TT::PL + cell] : 0u;
        f[i] = dec_pair<typename TT::Fmt>(i, b, tile[(qi - 1) * TT::PL + cell],
                        make_float2(ref[cell], ref[TT::PL + cell]), wx, wy);
    }
}

// FP16 storage: the 4 scaled solute populations (bb: the D2Q9 bounce-back
// bits; D2Q4 direction k is D2Q9 direction k + 1).
template <class TT, bool BB>
__device__ __forceinline__ void spull16s(const uint32_t *tile, int c,
                                         unsigned bb, float g[QS]) {
    const float *ref = reinterpret_cast<const float *>(tile) + (W16_REF + 2) * TT::PL;
#pragma unroll
    for (int k = 0; k < QS; ++k) {
        const bool b = BB && ((bb >> (k + 1)) & 1u);
        const int cell = b ? c : c - sy(k) * TT::BX - sx(k);
        const int qk = b ? sopp(k) : k;
        g[k] = dec_sol16<typename TT::Fmt>(tile[(W16_SOL + (qk >> 1)) * TT::PL + cell], qk,
                                           ref[cell]);
    }
}

// The 22 populations of the node at stage cell c, FP32 storage (fA, fB, g)
// or FP16 storage (scaled {A, B} pairs in fA2, solute in g).  `fast`
// (bb == 0 on every lane that calls) takes the path without bounce-back
// selects; the other path gives the same values for bb == 0, so a warp with
// any bounce-back lane runs that one alone.
template <class S, class TT>
__device__ __forceinline__ void spull22(const typename S::T *tile, int c,
                                        unsigned bb, bool fast, float fA[Q],
                                        float fB[Q], float2 fA2[Q],
                                        float g[QS]) {
    if constexpr (!S::kHalf) {
        if (fast) {
            spull9<TT, false>(tile, 0, c, 0u, fA);
            spull9<TT, false>(tile, 1, c, 0u, fB);
            spull4<TT, false>(tile, c, 0u, g);
        } else {
            spull9<TT, true>(tile, 0, c, bb, fA);
            spull9<TT, true>(tile, 1, c, bb, fB);
            spull4<TT, true>(tile, c, (bb >> 1) & 0xFu, g);
        }
    } else {
        if (fast) {
            spull16ab<TT, false>(tile, c, 0u, fA2);
            spull16s<TT, false>(tile, c, 0u, g);
        } else {
            spull16ab<TT, true>(tile, c, bb, fA2);
            spull16s<TT, true>(tile, c, bb, g);
        }
    }
}

// Densities of both components at stage cell c (`fast` as for spull22),
// formed as the node's own update forms them.
template <class S, class TT>
__device__ __forceinline__ float2 sdens(const typename S::T *tile, int c,
                                        unsigned bb, bool fast) {
    if constexpr (!S::kHalf) {
        float f[Q];
        float ra = 0.f, rb = 0.f;
        if (fast) {
            spull9<TT, false>(tile, 0, c, 0u, f);
#pragma unroll
            for (int i = 0; i < Q; ++i) ra += f[i];
            spull9<TT, false>(tile, 1, c, 0u, f);
#pragma unroll
            for (int i = 0; i < Q; ++i) rb += f[i];
        } else {
            spull9<TT, true>(tile, 0, c, bb, f);
#pragma unroll
            for (int i = 0; i < Q; ++i) ra += f[i];
            spull9<TT, true>(tile, 1, c, bb, f);
#pragma unroll
            for (int i = 0; i < Q; ++i) rb += f[i];
        }
        return make_float2(ra, rb);
    } else {
        float2 f[Q];
        if (fast)
            spull16ab<TT, false>(tile, c, 0u, f);
        else
            spull16ab<TT, true>(tile, c, bb, f);
        return dens2(f);
    }
}

// True when no node in rows ly - 1 .. ly + 1, columns c0 - 1 .. c0 + 32 of
// the tile (c0 = this warp's first column) has `bits` set in the mask box:
// then every node of the warp has no solid neighbour and no solid source.
// The 34 bytes of a row lie in 10 aligned words; lane j < 30 tests one.
template <class TT>
__device__ __forceinline__ bool warp_clean(const uint8_t *sm, int ly, int c0,
                                           int lane, uint8_t bits) {
    bool dirty = false;
    if (lane < 30) {
        const int row = lane / 10, w = lane % 10;
        const int off = (ly + 1 + row) * TT::MBX + TT::MXO + c0 - 4 + 4 * w;
        unsigned keep = 0xFFFFFFFFu;
        if (w == 0) keep = 0xFF000000u;  // column c0 - 1 only
        if (w == 9) keep = 0x000000FFu;  // column c0 + 32 only
        const unsigned v = *reinterpret_cast<const unsigned *>(sm + off);
        dirty = (v & keep & (bits * 0x01010101u)) != 0u;
    }
    return !__any_sync(0xFFFFFFFFu, dirty);
}

// Mask bits around the node at mask-box cell mc: bit i of the result is set
// when the node at mc + e_i (sign = +1) or mc - e_i (sign = -1) has `bit`.
template <class TT, int SIGN>
__device__ __forceinline__ unsigned nb_bits(const uint8_t *sm, int mc,
                                            uint8_t bit) {
    unsigned r = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (sm[mc + SIGN * (cy(i) * TT::MBX + cx(i))] & bit) r |= 1u << i;
    return r;
}

// Tensor maps of one launch, per lattice: the tile copies (populations,
// mask) and the output stores.
struct TmaMaps {
    const CUtensorMap *pop, *mask, *out;
};

// SUM: the launch also adds up the lattice totals (StepArgs::sums).
template <class S, int TX, int TY, bool SUM>
__global__ void __launch_bounds__(TX *TY, (TmaTile<S, TX, TY>::MINB))
    k_step_tma(StepArgs a, TmaMaps mp, const TileRec *__restrict__ sched,
               int nslots, int *__restrict__ err) {
    using TT = TmaTile<S, TX, TY>;
    using T = typename S::T;
    extern __shared__ __align__(128) unsigned char smem[];
    auto stage_pop = [&](int s) { return reinterpret_cast<T *>(smem + s * TT::STAGE); };
    auto stage_mask = [&](int s) { return smem + s * TT::STAGE + TT::MASK_OFF; };
    auto sdesc = [&](int slot) {
        return reinterpret_cast<LatDesc *>(smem + TT::DESC_OFF + 128 * slot);
    };
    auto srho = [&](int f) {
        return reinterpret_cast<float *>(smem + TT::RHO_OFF + f * TT::RHO_AL);
    };
    constexpr int NS = TT::NS, NSL = TT::NSL;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TT::BAR_OFF);  // NS
    long long *s_t = reinterpret_cast<long long *>(bar + 3);
    TileRec *s_rec = reinterpret_cast<TileRec *>(bar + 4);  // tile of each desc slot

    // This block's tiles: sched[blockIdx.x + k * gridDim.x], k = 0, 1, ...,
    // until the first -1; consecutive entries mostly walk down one tile
    // column of a lattice, so the halo rows a tile copies were copied by the
    // previous tile of the same block and come from L2.
    auto sched_at = [&](int k) {
        return k < nslots ? sched[blockIdx.x + (size_t)k * gridDim.x]
                          : TileRec{-1, 0, 0, 0};
    };

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;

    // Copies tile r into stage s and its lattice descriptor into `slot`.
    auto issue = [&](const TileRec &r, int s, int slot, int extra_tx) {
        const int l = r.lat;
        // physical coordinates: column x0 - XO and row y0 - 2 of the lattice
        const int x0 = r.x0 + XGHOST;
        const int y0 = r.y0;
        fence_proxy_async();
        mbar_expect_tx(&bar[s], TT::TX_BYTES + extra_tx);
        bulk_load(sdesc(slot), a.desc + l, 128, &bar[s]);
        tma_load_3d(stage_pop(s), &mp.pop[l], x0 - TT::XO, y0, 0, &bar[s]);
        tma_load_2d(stage_mask(s), &mp.mask[l], x0 - TT::MXO, y0, &bar[s]);
    };

    if (tid == 0) {
        for (int j = 0; j < NS; ++j) mbar_init(&bar[j], 1);
        fence_mbar_init();
        *s_t = *(volatile long long *)a.step;
        bool more = true;
        for (int j = 0; j < NSL; ++j) {
            const TileRec r = more && j < NS ? sched_at(j) : TileRec{-1, 0, 0, 0};
            s_rec[j] = r;
            more = r.lat >= 0;
            // (the test hook: block 0's first tile waits for bytes that
            // never come, so its bounded wait runs out)
            if (more) issue(r, j, j, j == 0 && blockIdx.x == 0 ? a.stall_tx : 0);
        }
    }
    __syncthreads();
    const long long t = *s_t;
    const MaskBits mb(t);

    // output tiles in shared memory (TS): node lid = ly * TX + lx of plane q
    // at sout(b)[q * NT + lid]
    auto sout = [&](int b) {
        return reinterpret_cast<T *>(smem + TT::OUT_OFF +
                                     (TT::NOUT == 2 ? (b & 1) : 0) * TT::OUT_BYTES);
    };
    // bulk tensor store of output tile b (thread 0; every thread fenced its
    // writes and passed a barrier since)
    auto store_out = [&](const TileRec &r, int b) {
        tma_store_3d(&mp.out[r.lat], sout(b), r.x0, r.y0, 0);
        bulk_commit();
    };
    // thread 0: the tile whose output awaits its store, and its output tile
    TileRec prev{-1, 0, 0, 0};
    int prev_buf = 0;
    bool failed = false;
    // gives up after a bounded wait ran out: lets the copies still in
    // flight land before exiting
    auto give_up = [&](int k, unsigned par) {
        if (tid == 0) {
            atomicOr(err, 1);
            for (int j = 1; j < NS; ++j) {
                if (s_rec[(k + j) % NSL].lat < 0) break;
                const int sj = (k + j) % NS;
                mbar_wait_bounded(&bar[sj], (par >> sj) & 1u);
            }
        }
    };

    unsigned parity = 0u;  // bit s: phase parity of stage s
    TotAcc acc;
    if constexpr (SUM) tot_reset(acc, -1);
    for (int k = 0; s_rec[k % NSL].lat >= 0; ++k) {
        // the record of the tile NS ahead, fetched now so that its load
        // latency hides behind this tile's work
        TileRec nxt{-1, 0, 0, 0};
        if (tid == 0 && s_rec[(k + NS - 1) % NSL].lat >= 0) nxt = sched_at(k + NS);
        const int s = k % NS;
        const int slot = k % NSL;
        const bool ok = mbar_wait_bounded(&bar[s], (parity >> s) & 1u);
        parity ^= 1u << s;
        if constexpr (!TT::ONE_BAR) {
            if (__syncthreads_or(!ok)) {
                give_up(k, parity);
                failed = true;
                break;
            }
            // every thread finished the previous tile's output
            if (TT::TS && tid == 0 && prev.lat >= 0) store_out(prev, 0);
        }
        // (ONE_BAR: a thread whose wait ran out still reads the stage --
        // shared memory at fixed offsets, results discarded -- and the
        // failure is taken at the barrier below)
        const TileRec rc = s_rec[slot];
        const LatDesc &d = *sdesc(slot);
        const int l = rc.lat;
        const int nx = d.nx, ny = d.ny;
        const int tx0 = rc.x0, ty0 = rc.y0;
        // rows / columns of the tile that hold lattice nodes; frame
        // positions further out are never a node's neighbour
        const int n_act = min(TY, ny - ty0), m_act = min(TX, nx - tx0);
        T *tp = stage_pop(s);
        uint8_t *sm = stage_mask(s);

        // own node: mask bits, pull, density
        const int lx = tid % TX, ly = tid / TX;
        const int x = tx0 + lx, y = ty0 + ly;
        const bool active = (x < nx) && (y < ny);
        const bool in_frame = lx <= m_act && ly <= n_act;  // neighbour of a node
        const int pc = (ly + 2) * TT::BX + lx + TT::XO;    // stage cell
        const int mc = (ly + 2) * TT::MBX + lx + TT::MXO;  // mask cell
        const uint8_t s_own = in_frame ? sm[mc] : (uint8_t)0xFF;
        const bool own_pull_fluid = !(s_own & mb.pull);
        // warps whose rows and their neighbours hold no solid node skip the
        // neighbour bits (all zero) and the bounce-back selects
        const bool clean = warp_clean<TT>(sm, ly, lx & ~31, lane,
                                          (uint8_t)(mb.pull | mb.force));
        const unsigned bb = clean ? 0u : nb_bits<TT, -1>(sm, mc, mb.pull);   // sources solid
        const unsigned snb = clean ? 0u : nb_bits<TT, +1>(sm, mc, mb.force); // neighbours solid
        float fA[Q], fB[Q], g[QS];
        float2 f2[Q];  // FP16 storage: scaled {A, B} pairs
        float *fr = srho(k & 1);
        float2 rho = make_float2(0.f, 0.f);
        {
            if (own_pull_fluid) {
                spull22<S, TT>(tp, pc, bb, clean, fA, fB, f2, g);
                if constexpr (S::kHalf) {
                    rho = dens2(f2);
                } else {
#pragma unroll
                    for (int i = 0; i < Q; ++i) { rho.x += fA[i]; rho.y += fB[i]; }
                }
            }
            const bool force_solid = s_own & mb.force;
            const int fc = (ly + 1) * TT::RX + lx + 1;
            if constexpr (S::kHalf) {
                reinterpret_cast<float2 *>(fr)[fc] =
                    force_solid ? make_float2(0.f, 0.f) : rho;
            } else {
                fr[fc] = force_solid ? 0.f : rho.x;
                fr[TT::RX * TT::RY + fc] = force_solid ? 0.f : rho.y;
            }
        }
        // ring of the density frame: the lanes of the first warps take
        // RW consecutive ring cells each (consecutive addresses, no
        // shared-memory bank conflicts).  FP16 storage: when the previous
        // tile of this block is the one just above (a strip walks down a
        // tile column), the top ring row is that tile's last frame row
        // (its last row of nodes and their side ring cells, same step),
        // copied instead of pulled again.
        {
            const TileRec rp = s_rec[(k + NSL - 1) % NSL];
            const bool above = S::kHalf && k > 0 && rp.lat == rc.lat &&
                               rp.x0 == tx0 && rp.y0 + TY == ty0;
            const int r = warp * TT::RW + lane;
            if (lane < TT::RW && r < TT::NRING) {
                int ry, rx;
                if (r < TT::RX) { ry = 0; rx = r; }
                else if (r < 2 * TT::RX) { ry = TT::RY - 1; rx = r - TT::RX; }
                else if (r < 2 * TT::RX + TY) { ry = 1 + r - 2 * TT::RX; rx = 0; }
                else { ry = 1 + r - 2 * TT::RX - TY; rx = TT::RX - 1; }
                const int rmc = (ry + 1) * TT::MBX + rx - 1 + TT::MXO;
                const int rpc = (ry + 1) * TT::BX + rx - 1 + TT::XO;
                float2 q = make_float2(0.f, 0.f);
                if (above && ry == 0) {
                    q = reinterpret_cast<const float2 *>(srho((k + 1) & 1))[TY * TT::RX + rx];
                } else if (!(sm[rmc] & mb.force)) {
                    // per lane: a warp-uniform choice here measured slower
                    const unsigned rbb = nb_bits<TT, -1>(sm, rmc, mb.pull);
                    q = sdens<S, TT>(tp, rpc, rbb, rbb == 0u);
                }
                const int fc = ry * TT::RX + rx;
                if constexpr (S::kHalf) {
                    reinterpret_cast<float2 *>(fr)[fc] = q;
                } else {
                    fr[fc] = q.x;
                    fr[TT::RX * TT::RY + fc] = q.y;
                }
            }
        }
        fence_proxy_async();
        // Output through shared memory and a bulk tensor store, except for
        // tiles that end past the lattice's last column: a store box that
        // crosses x = nx was measured to overwrite the ghost columns there
        // (partial 16-byte rows are not clipped element by element), so
        // those tiles store their nodes directly.
        const bool ts_tile = TT::TS && tx0 + TX <= nx;
        if constexpr (TT::TS) {
            // the output tile written below must have been read by its last
            // store (ONE_BAR: the store of two tiles ago)
            if (tid == 0) bulk_wait_read();
        }
        if constexpr (TT::ONE_BAR) {
            if (__syncthreads_or(!ok)) {
                give_up(k, parity);
                failed = true;
                break;
            }
            // every thread finished the previous tile's output
            if (tid == 0) {
                if (prev.lat >= 0) store_out(prev, prev_buf);
                prev = ts_tile ? rc : TileRec{-1, 0, 0, 0};
                prev_buf = k & 1;
            }
        } else {
            if (TT::TS && tid == 0) prev = ts_tile ? rc : TileRec{-1, 0, 0, 0};
            __syncthreads();
        }
        // stage s is free: start the copy of the tile NS ahead into it
        if (tid == 0) {
            s_rec[(k + NS) % NSL] = nxt;
            if (nxt.lat >= 0) issue(nxt, s, (k + NS) % NSL, 0);
        }

        constexpr bool want = SUM;
        NodeTot tot{0.f, 0.f, 0.f};
        if (active) {
            const int own = y * d.pitch + x;
            const int lid = ly * TX + lx;
            if (s_own & mb.force) {
                if (own_pull_fluid) {
                    if constexpr (S::kHalf)
                        retire_node16(a, d, l, own, f2, g);
                    else
                        retire_node(a, d, l, own, fA, fB, g);
                }
                const uint8_t nb = s_own | mb.next;
                if (nb != s_own) mask_store(a.mask + d.node_off, own, x, y, nx, ny, d.pitch, nb);
            } else {
                const int ns = __popc(snb & 0x1Eu);
                bool flagged;
                if constexpr (S::kHalf) {
                    float2 nbv[Q];
#pragma unroll
                    for (int i = 1; i < Q; ++i)
                        nbv[i] = reinterpret_cast<const float2 *>(fr)[
                            (ly + 1 + cy(i)) * TT::RX + lx + 1 + cx(i)];
                    flagged = fluid_update16<typename S::Fmt>(
                        a, d, l, t, x, y, own, f2, g, rho, nbv, snb, ns,
                        [&](const uint32_t *v) {
                            if (ts_tile)
                                store_words16(sout(k) + lid, TT::NT, v);
                            else
                                store_words16(static_cast<uint32_t *>(a.fout) +
                                                  d.pop_off + own,
                                              (int)d.plane, v);
                        },
                        want, tot);
                } else {
                    float rAn[Q], rBn[Q];
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const int fc = (ly + 1 + cy(i)) * TT::RX + lx + 1 + cx(i);
                        rAn[i] = fr[fc];
                        rBn[i] = fr[TT::RX * TT::RY + fc];
                    }
                    flagged = fluid_update(
                        a, d, l, t, x, y, own, fA, fB, g, rAn, rBn, snb, ns,
                        [&](const float *pa, const float *pb, const float *pg) {
                            if (ts_tile)
                                store22_f32(reinterpret_cast<float *>(sout(k)) + lid,
                                            TT::NT, pa, pb, pg);
                            else
                                store_node22(a, d, own, pa, pb, pg);
                        },
                        want, tot);
                }
                if (flagged)
                    mask_store(a.mask + d.node_off, own, x, y, nx, ny, d.pitch, s_own | mb.next);
            }
        }
        if constexpr (SUM) tot_add(acc, tot, l, a.sums, lane);
        if constexpr (TT::TS) fence_proxy_async();  // before the next barrier
    }
    if constexpr (TT::TS) {
        __syncthreads();
        if (tid == 0) {
            if (!failed && prev.lat >= 0) store_out(prev, prev_buf);
            bulk_wait_all();
        }
    }
    if constexpr (SUM) tot_flush(acc, a.sums, lane);
    finish_launch(a, t);
}

// ---- host side ---------------------------------------------------------------

template <class S, int TX, int TY>
static cudaError_t grid_tma_t(int *grid) {
    using TT = TmaTile<S, TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(
        k_step_tma<S, TX, TY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        TT::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step_tma<S, TX, TY, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TT::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_tma<S, TX, TY, false>,
                                                      TX * TY, TT::SMEM);
    if (e != cudaSuccess) return e;
    *grid = sms * (per > 0 ? per : 1);
    return cudaSuccess;
}

template <class S, int TX, int TY>
static cudaError_t launch_tma_t(const StepArgs &a, const TmaMaps &mp,
                                const TileRec *sched, int nslots, int grid,
                                int *err, cudaStream_t s) {
    using TT = TmaTile<S, TX, TY>;
    if (a.sums)
        k_step_tma<S, TX, TY, true><<<grid, TX * TY, TT::SMEM, s>>>(a, mp, sched,
                                                                    nslots, err);
    else
        k_step_tma<S, TX, TY, false><<<grid, TX * TY, TT::SMEM, s>>>(a, mp, sched,
                                                                     nslots, err);
    return cudaGetLastError();
}

#define LBM_TMA_SHAPES(M) M(32, 8) M(32, 4) M(64, 4) M(32, 16) M(64, 8) M(128, 4)

// Persistent grid of the TMA step kernel for a tile shape (also sets its
// shared-memory limit); 0 on an unsupported shape.
// store: 0 FP32, 1 FP16, 2 BF16 storage
cudaError_t grid_step_tma(int tx, int ty, int store, int *grid) {
    *grid = 0;
#define LBM_TMA_GRID(X, Y)                                                   \
    if (tx == X && ty == Y)                                                  \
        return store == 2   ? grid_tma_t<Store16<BF16>, X, Y>(grid)          \
               : store == 1 ? grid_tma_t<Store16<F16>, X, Y>(grid)           \
                            : grid_tma_t<Store32, X, Y>(grid);
    LBM_TMA_SHAPES(LBM_TMA_GRID)
#undef LBM_TMA_GRID
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_tma(const StepArgs &a, const CUtensorMap *pop_maps,
                            const CUtensorMap *mask_maps,
                            const CUtensorMap *out_maps, const TileRec *sched,
                            int nslots, int grid, int tx, int ty, int store,
                            int *err, cudaStream_t s) {
    const TmaMaps mp{pop_maps, mask_maps, out_maps};
#define LBM_TMA_CASE(X, Y)                                                   \
    if (tx == X && ty == Y)                                                  \
        return store == 2                                                    \
                   ? launch_tma_t<Store16<BF16>, X, Y>(a, mp, sched, nslots, \
                                                       grid, err, s)         \
               : store == 1                                                  \
                   ? launch_tma_t<Store16<F16>, X, Y>(a, mp, sched, nslots,  \
                                                      grid, err, s)          \
                   : launch_tma_t<Store32, X, Y>(a, mp, sched, nslots, grid, \
                                                 err, s);
    LBM_TMA_SHAPES(LBM_TMA_CASE)
#undef LBM_TMA_CASE
    return cudaErrorInvalidValue;
}

// Tensor map geometry must match TmaTile: box (TX + 8) x (TY + 4) x
// planes of 32-bit words for the populations, (TX + 32) x (TY + 4) for the
// mask; the output maps span the lattice itself with box TX x TY x planes.
int tma_box_x(int tx) { return tx + 8; }
int tma_mask_box_x(int tx) { return tx + 32; }

}  // namespace lbmk
