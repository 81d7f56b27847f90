// lbm_step.cu -- the fused reactive lattice Boltzmann time step (sm_103a).
//
// One launch advances every lattice of a handle by one step.  A block owns
// a TX x TY tile of one lattice and does, per node, the whole step of the
// paper's Sec. II model in one pass over HBM:
//   1. pull-streaming with half-way bounce-back of the 9 + 9 populations
//      (each read once), giving the post-streaming state of this step;
//   2. densities of the tile plus a one-node ring (the ring's pulls are
//      L2 hits: neighbouring tiles read the same lines), kept in shared
//      memory for the cohesion stencil;
//   3. Martys-Chen cohesion and adhesion forces, Shan-Chen velocity shift,
//      BGK collision of both components;
//   4. pull of the D2Q4 solute, its BGK collision with the barycentric
//      velocity (inlet column imposed), first-order surface reaction;
//   5. FP64 deposit update and threshold test; a node that reaches it is
//      flagged in the mask (turns solid for the next step's forces, keeps
//      the streaming of this step -- see MaskBits);
//   6. a node flagged in the previous step hands its post-streaming fluid,
//      solute and deposit to the lattice ledger instead of colliding.
// The solid mask and the deposit are read only as a byte per node and a
// double per reacting node; populations of solid nodes are never touched.
//
// Floating point: FP32 arithmetic in the order of the collision formulas;
// the deposit and its threshold test are FP64.  Populations are stored as
// FP32 (Store32) or as FP16 deviations from FP32 references (Store16, see
// lbm_device.cuh).
#include "lbm_node.cuh"

namespace lbmk {

template <int TX, int TY>
struct Tile {
    static constexpr int NT = TX * TY;
    static constexpr int HX = TX + 4, HY = TY + 4;  // mask halo, radius 2
    static constexpr int RX = TX + 2, RY = TY + 2;  // density frame, radius 1
    static constexpr int NRING = 2 * RX + 2 * TY;
};

// Bounce-back bits of the 9 pulls of the node at mask-halo slot (hy, hx):
// bit i set when the source x - e_i was solid for the streaming.
template <int HX>
__device__ __forceinline__ unsigned pull_bits(const uint8_t (*sm)[HX], int hy,
                                              int hx, uint8_t pullbit) {
    unsigned bb = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (sm[hy - cy(i)][hx - cx(i)] & pullbit) bb |= 1u << i;
    return bb;
}

// Pulls the 9 populations of component `comp` into node (gx, gy), FP32
// storage.
__device__ __forceinline__ void pull9(const float *__restrict__ fin,
                                      const LatDesc &d, int comp, int gx,
                                      int gxm, int gxp, int gy, int gym,
                                      int gyp, unsigned bb, float f[Q]) {
    const int64_t own = (int64_t)gy * d.pitch + gx;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sxx = cx(i) > 0 ? gxm : (cx(i) < 0 ? gxp : gx);
        const int syy = cy(i) > 0 ? gym : (cy(i) < 0 ? gyp : gy);
        const bool b = (bb >> i) & 1u;
        const int64_t src = b ? own : (int64_t)syy * d.pitch + sxx;
        const int qi = b ? opp(i) : i;
        f[i] = __ldg(fin + d.pop_off + (comp * Q + qi) * d.plane + src);
    }
}

// Pulls the 4 solute populations into node (gx, gy), FP32 storage;
// bounce-back where the D2Q4 source was solid.
__device__ __forceinline__ void pull4(const float *__restrict__ fin,
                                      const LatDesc &d, int gx, int gxm,
                                      int gxp, int gy, int gym, int gyp,
                                      unsigned bb4, float g[QS]) {
    const int64_t own = (int64_t)gy * d.pitch + gx;
#pragma unroll
    for (int k = 0; k < QS; ++k) {
        const int sxx = sx(k) > 0 ? gxm : (sx(k) < 0 ? gxp : gx);
        const int syy = sy(k) > 0 ? gym : (sy(k) < 0 ? gyp : gy);
        const bool b = (bb4 >> k) & 1u;
        const int64_t src = b ? own : (int64_t)syy * d.pitch + sxx;
        g[k] = __ldg(fin + d.pop_off + (2 * Q + (b ? sopp(k) : k)) * d.plane + src);
    }
}

// 16-bit storage (format F): the scaled {A, B} populations pulled into
// node (gx, gy) (bb: bounce-back bits of the 9 directions).
template <class F>
__device__ __forceinline__ void pull16ab(const uint32_t *__restrict__ fin,
                                         const LatDesc &d, int gx, int gxm,
                                         int gxp, int gy, int gym, int gyp,
                                         unsigned bb, float2 f[Q]) {
    const uint32_t *w = fin + d.pop_off;
    const float *ref = reinterpret_cast<const float *>(w + W16_REF * d.plane);
    const int64_t own = (int64_t)gy * d.pitch + gx;
    f[0] = make_float2(__ldg(ref + own), __ldg(ref + d.plane + own));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int sxx = cx(i) > 0 ? gxm : (cx(i) < 0 ? gxp : gx);
        const int syy = cy(i) > 0 ? gym : (cy(i) < 0 ? gyp : gy);
        const bool b = (bb >> i) & 1u;
        const int64_t src = b ? own : (int64_t)syy * d.pitch + sxx;
        const int qi = b ? opp(i) : i;
        const uint32_t wx = cx(i) != 0 ? __ldg(w + W16_VEL * d.plane + src) : 0u;
        const uint32_t wy = cy(i) != 0 ? __ldg(w + (W16_VEL + 1) * d.plane + src) : 0u;
        f[i] = dec_pair<F>(i, b, __ldg(w + (qi - 1) * d.plane + src),
                        make_float2(__ldg(ref + src), __ldg(ref + d.plane + src)),
                        wx, wy);
    }
}

// FP16 storage: the 4 scaled solute populations of node (gx, gy) (bb4:
// bounce-back bits of the 4 directions).
template <class F>
__device__ __forceinline__ void pull16s(const uint32_t *__restrict__ fin,
                                        const LatDesc &d, int gx, int gxm,
                                        int gxp, int gy, int gym, int gyp,
                                        unsigned bb4, float g[QS]) {
    const uint32_t *w = fin + d.pop_off;
    const float *ref = reinterpret_cast<const float *>(w + (W16_REF + 2) * d.plane);
    const int64_t own = (int64_t)gy * d.pitch + gx;
#pragma unroll
    for (int k = 0; k < QS; ++k) {
        const int sxx = sx(k) > 0 ? gxm : (sx(k) < 0 ? gxp : gx);
        const int syy = sy(k) > 0 ? gym : (sy(k) < 0 ? gyp : gy);
        const bool b = (bb4 >> k) & 1u;
        const int64_t src = b ? own : (int64_t)syy * d.pitch + sxx;
        const int qk = b ? sopp(k) : k;
        g[k] = dec_sol16<F>(__ldg(w + (W16_SOL + (qk >> 1)) * d.plane + src), qk,
                         __ldg(ref + src));
    }
}

// Both components' populations and their densities {rho_A, rho_B}, as the
// TMA kernel forms them: FP32 storage into fA, fB; FP16 storage as scaled
// {A, B} pairs into f2.
template <class S>
__device__ __forceinline__ float2 pull_ab(const StepArgs &a, const LatDesc &d,
                                          int gx, int gxm, int gxp, int gy,
                                          int gym, int gyp, unsigned bb,
                                          float fA[Q], float fB[Q],
                                          float2 f2[Q]) {
    if constexpr (!S::kHalf) {
        const float *fin = static_cast<const float *>(a.fin);
        pull9(fin, d, 0, gx, gxm, gxp, gy, gym, gyp, bb, fA);
        pull9(fin, d, 1, gx, gxm, gxp, gy, gym, gyp, bb, fB);
        float ra = 0.f, rb = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) { ra += fA[i]; rb += fB[i]; }
        return make_float2(ra, rb);
    } else {
        pull16ab<typename S::Fmt>(static_cast<const uint32_t *>(a.fin), d, gx,
                                  gxm, gxp, gy, gym, gyp, bb, f2);
        return dens2(f2);
    }
}

template <class S>
__device__ __forceinline__ void pull_sol(const StepArgs &a, const LatDesc &d,
                                         int gx, int gxm, int gxp, int gy,
                                         int gym, int gyp, unsigned bb4,
                                         float g[QS]) {
    if constexpr (!S::kHalf)
        pull4(static_cast<const float *>(a.fin), d, gx, gxm, gxp, gy, gym, gyp,
              bb4, g);
    else
        pull16s<typename S::Fmt>(static_cast<const uint32_t *>(a.fin), d, gx,
                                 gxm, gxp, gy, gym, gyp, bb4, g);
}

// SUM: the launch also adds up the lattice totals (StepArgs::sums).
template <class S, int TX, int TY, bool SUM>
__global__ void __launch_bounds__(TX *TY)
    k_step(StepArgs a) {
    using TL = Tile<TX, TY>;
    __shared__ uint8_t smask[TL::HY][TL::HX];
    __shared__ float srho[2][TL::RY][TL::RX];
    __shared__ long long s_t;

    const int tid = threadIdx.x;
    const int l = a.tile_lat[blockIdx.x];
    const LatDesc d = a.desc[l];
    const int nx = d.nx, ny = d.ny;
    const int local = blockIdx.x - d.tile_base;
    const int tx0 = (local % d.tiles_x) * TX;
    const int ty0 = (local / d.tiles_x) * TY;
    uint8_t *__restrict__ mask = a.mask + d.node_off;

    if (tid == 0) s_t = *(volatile long long *)a.step;
    for (int k = tid; k < TL::HY * TL::HX; k += TL::NT) {
        const int hy = k / TL::HX, hx = k - hy * TL::HX;
        const int gy = wrapg(ty0 - 2 + hy, ny), gx = wrapg(tx0 - 2 + hx, nx);
        smask[hy][hx] = mask[(int64_t)gy * d.pitch + gx];
    }
    __syncthreads();
    const long long t = s_t;
    const MaskBits mb(t);

    // --- own node: pull and density --------------------------------------
    const int lx = tid % TX, ly = tid / TX;
    const int x = tx0 + lx, y = ty0 + ly;
    const bool active = (x < nx) && (y < ny);
    const int gx = wrapg(x, nx), gy = wrapg(y, ny);
    const int gxm = wrap1(gx - 1, nx), gxp = wrap1(gx + 1, nx);
    const int gym = wrap1(gy - 1, ny), gyp = wrap1(gy + 1, ny);
    const uint8_t s_own = smask[ly + 2][lx + 2];
    const bool own_pull_fluid = !(s_own & mb.pull);
    float fA[Q], fB[Q];
    float2 f2[Q];  // FP16 storage: scaled {A, B} pairs
    float2 rho = make_float2(0.f, 0.f);
    {
        if (own_pull_fluid) {
            const unsigned bb = pull_bits<TL::HX>(smask, ly + 2, lx + 2, mb.pull);
            rho = pull_ab<S>(a, d, gx, gxm, gxp, gy, gym, gyp, bb, fA, fB, f2);
        }
        const bool force_solid = s_own & mb.force;
        srho[0][ly + 1][lx + 1] = force_solid ? 0.f : rho.x;
        srho[1][ly + 1][lx + 1] = force_solid ? 0.f : rho.y;
    }
    // --- ring of the density frame ----------------------------------------
    for (int r = tid; r < TL::NRING; r += TL::NT) {
        int ry, rx;
        if (r < TL::RX) { ry = 0; rx = r; }
        else if (r < 2 * TL::RX) { ry = TL::RY - 1; rx = r - TL::RX; }
        else if (r < 2 * TL::RX + TY) { ry = 1 + r - 2 * TL::RX; rx = 0; }
        else { ry = 1 + r - 2 * TL::RX - TY; rx = TL::RX - 1; }
        const uint8_t s = smask[ry + 1][rx + 1];
        float2 q = make_float2(0.f, 0.f);
        if (!(s & mb.force)) {
            const int X = wrapg(tx0 - 1 + rx, nx), Y = wrapg(ty0 - 1 + ry, ny);
            const int Xm = wrap1(X - 1, nx), Xp = wrap1(X + 1, nx);
            const int Ym = wrap1(Y - 1, ny), Yp = wrap1(Y + 1, ny);
            const unsigned bb = pull_bits<TL::HX>(smask, ry + 1, rx + 1, mb.pull);
            float f[Q], h[Q];
            float2 p2[Q];
            q = pull_ab<S>(a, d, X, Xm, Xp, Y, Ym, Yp, bb, f, h, p2);
        }
        srho[0][ry][rx] = q.x;
        srho[1][ry][rx] = q.y;
    }
    __syncthreads();

    constexpr bool want = SUM;
    NodeTot tot{0.f, 0.f, 0.f};
    if (active) {
        const int own = gy * d.pitch + gx;
        const int hy = ly + 2, hx = lx + 2;
        unsigned bb4 = 0;
        int ns = 0;
#pragma unroll
        for (int k = 0; k < QS; ++k) {
            if (smask[hy - sy(k)][hx - sx(k)] & mb.pull) bb4 |= 1u << k;
            if (smask[hy + sy(k)][hx + sx(k)] & mb.force) ++ns;
        }
        if (s_own & mb.force) {
            const uint8_t nb = s_own | mb.next;
            if (own_pull_fluid) {
                float g[QS];
                pull_sol<S>(a, d, gx, gxm, gxp, gy, gym, gyp, bb4, g);
                if constexpr (S::kHalf)
                    retire_node16(a, d, l, own, f2, g);
                else
                    retire_node(a, d, l, own, fA, fB, g);
            }
            if (nb != s_own) mask_store(mask, own, gx, gy, nx, ny, d.pitch, nb);
        } else {
            float g[QS], rAn[Q], rBn[Q];
            unsigned snb = 0;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                rAn[i] = srho[0][ly + 1 + cy(i)][lx + 1 + cx(i)];
                rBn[i] = srho[1][ly + 1 + cy(i)][lx + 1 + cx(i)];
                if (smask[hy + cy(i)][hx + cx(i)] & mb.force) snb |= 1u << i;
            }
            pull_sol<S>(a, d, gx, gxm, gxp, gy, gym, gyp, bb4, g);
            bool flagged;
            if constexpr (S::kHalf) {
                float2 nbv[Q];
#pragma unroll
                for (int i = 1; i < Q; ++i) nbv[i] = make_float2(rAn[i], rBn[i]);
                flagged = fluid_update16<typename S::Fmt>(
                    a, d, l, t, gx, gy, own, f2, g, rho, nbv, snb, ns,
                    [&](const uint32_t *v) {
                        store_words16(static_cast<uint32_t *>(a.fout) + d.pop_off + own,
                                      (int)d.plane, v);
                    },
                    want, tot);
            } else {
                flagged = fluid_update(
                    a, d, l, t, gx, gy, own, fA, fB, g, rAn, rBn, snb, ns,
                    [&](const float *pa, const float *pb, const float *pg) {
                        store_node22(a, d, own, pa, pb, pg);
                    },
                    want, tot);
            }
            if (flagged) mask_store(mask, own, gx, gy, nx, ny, d.pitch, s_own | mb.next);
        }
    }
    if constexpr (SUM) {
        TotAcc acc;
        tot_reset(acc, l);
        tot_add(acc, tot, l, a.sums, tid & 31);
        tot_flush(acc, a.sums, tid & 31);
    }
    finish_launch(a, t);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <int TX, int TY, bool SUM>
static void launch_tile_t(const StepArgs &a, int ntiles, int store,
                          cudaStream_t s) {
    if (store == 2)
        k_step<Store16<BF16>, TX, TY, SUM><<<ntiles, TX * TY, 0, s>>>(a);
    else if (store == 1)
        k_step<Store16<F16>, TX, TY, SUM><<<ntiles, TX * TY, 0, s>>>(a);
    else
        k_step<Store32, TX, TY, SUM><<<ntiles, TX * TY, 0, s>>>(a);
}

template <int TX, int TY>
static cudaError_t launch_tile(const StepArgs &a, int ntiles, int store,
                               cudaStream_t s) {
    if (a.sums)
        launch_tile_t<TX, TY, true>(a, ntiles, store, s);
    else
        launch_tile_t<TX, TY, false>(a, ntiles, store, s);
    return cudaGetLastError();
}

// store: 0 FP32, 1 FP16, 2 BF16 storage
cudaError_t launch_step_direct(const StepArgs &a, int ntiles, int tx,
                               int ty, int store, cudaStream_t s) {
    if (tx == 32 && ty == 8) return launch_tile<32, 8>(a, ntiles, store, s);
    if (tx == 32 && ty == 4) return launch_tile<32, 4>(a, ntiles, store, s);
    if (tx == 32 && ty == 16) return launch_tile<32, 16>(a, ntiles, store, s);
    if (tx == 64 && ty == 4) return launch_tile<64, 4>(a, ntiles, store, s);
    if (tx == 64 && ty == 8) return launch_tile<64, 8>(a, ntiles, store, s);
    if (tx == 128 && ty == 4) return launch_tile<128, 4>(a, ntiles, store, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbmk
