// lbm_device.cuh -- device-side layout and lattice constants of the
// reactive two-component lattice Boltzmann library (sm_103a).
//
// Layout in HBM (one handle, `count` lattices packed back to back):
//   populations: two ping-pong buffers; in each, lattice l owns 22
//     consecutive planes of (ny + 4) * pitch elements (A: 9, B: 9, solute:
//     4), rows padded to `pitch` (a multiple of 32 elements, so every row
//     starts on a 128-byte boundary in FP32 storage);
//   FP16 storage keeps 20 FP16 planes per lattice (the 8 moving A and 8
//     moving B populations, then the 4 solute ones, see sp16) and, per
//     lattice and buffer, a moment block of 5 FP16 reference planes
//     (w_1 rho~ and w_5 rho~ of A and of B, C~ / 4, see refp) followed by
//     2 FP32 planes holding the rest populations of A and B (rest_planes);
//   every plane (populations, moments, mask) has a two-node ghost band
//     around the lattice -- rows -2, -1, ny, ny + 1 and columns -2, -1, nx,
//     nx + 1 -- holding the periodic images of the nodes next to the
//     boundaries; the offsets below point at logical node (0, 0), which
//     sits at physical row 2 and column 16 of the lattice's planes, so node
//     (x, y) is at offset y * pitch + x for -2 <= x < nx + 2,
//     -2 <= y < ny + 2; the nodes next to the boundaries refresh their
//     images whenever they write;
//   mask: one byte per node, read and written in place (see MaskBits);
//   deposit: one double per node;
//   per section column: fluid-node counter (closure), initial wall
//     thickness below and above (observables);
//   per lattice: ledgers, closure step, non-finite flag.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbmk {

constexpr int Q = 9;      // D2Q9 per fluid component
constexpr int QS = 4;     // D2Q4 solute
constexpr int NPOP = 22;  // 9 + 9 + 4 planes per lattice
constexpr int NMOM = 5;   // FP16 storage: reference planes (see refp)
constexpr int NP16 = 20;  // FP16 storage: population planes (no rest ones)
constexpr int NREST = 2;  // FP16 storage: FP32 rest planes of A and B
// FP16 storage: the moment block of a lattice spans 9 half-planes, the 5
// FP16 references then the 2 FP32 rest planes
constexpr int MOM_BLOCK = NMOM + 2 * NREST;

// FP16 storage plane of population q (A: 1..8, B: 10..17, solute 18..21;
// the rest populations 0 and 9 are FP32, in the moment block)
__host__ __device__ constexpr int sp16(int q) { return q < Q ? q - 1 : q - 2; }
// FP16 storage reference plane of moving population i (1..8) of component
// comp: w_1 rho~ and w_5 rho~ of A (planes 0, 1) and of B (2, 3); the
// solute's C~ / 4 is plane kSolRef
__host__ __device__ constexpr int refp(int comp, int i) { return 2 * comp + (i >= 5 ? 1 : 0); }
constexpr int kSolRef = 4;

// D2Q9 order (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
__host__ __device__ __forceinline__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
__host__ __device__ __forceinline__ constexpr float wq(int i) {
    return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// D2Q4 order (1,0) (0,1) (-1,0) (0,-1).
__host__ __device__ __forceinline__ constexpr int sx(int k) {
    return k == 0 ? 1 : (k == 2 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int sy(int k) {
    return k == 1 ? 1 : (k == 3 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int sopp(int k) { return (k + 2) & 3; }

// The mask byte keeps the solid set of three consecutive steps in three
// rotating bits.  Before the kernel of step t (t steps completed) runs, bit
// t%3 holds s_t (the solid set the forces, adhesion and reaction of step t
// see) and bit (t+2)%3 holds s_{t-1} (the set the streaming that ends step
// t-1 used, which the pull of step t replays).  Step t writes s_{t+1} into
// bit (t+1)%3, which held s_{t-2}: no reader of step t looks at that bit,
// so the in-place update is race free, and since solid only grows a node's
// byte changes on at most three steps after it is flagged.
struct MaskBits {
    uint8_t force, pull, next;
    __host__ __device__ explicit MaskBits(int64_t t) {
        int p = (int)(t % 3);
        force = (uint8_t)(1u << p);
        pull = (uint8_t)(1u << ((p + 2) % 3));
        next = (uint8_t)(1u << ((p + 1) % 3));
    }
};

// One lattice of the batch (128 bytes: the TMA step kernel bulk-copies it
// into shared memory next to each tile).
struct alignas(16) LatDesc {
    int32_t nx, ny, pitch, tiles_x;  // pitch >= nx + 2 * XGHOST
    int32_t tile_base, cap_x0, cap_x1, inlet;
    int64_t node_off;   // first node of this lattice in mask / deposit
    int64_t pop_off;    // first element of plane 0 in a population buffer
    int64_t mom_off;    // first element of moment plane 0 (FP16 storage)
    int64_t plane;      // (ny + 4) * pitch: rows -2 .. ny + 1
    int64_t col_off;    // first section column in per-column arrays
    float tau_a, tau_b, inv_tau_a, inv_tau_b, inv_tau_d;
    float g_coh, g_ads, k_r, c_in, body_x;
    double m_th;
    int32_t index;      // position of this lattice in the batch
    int32_t pad_;
};
static_assert(sizeof(LatDesc) == 128, "LatDesc is copied as 128 bytes");

// One tile of the persistent TMA kernel's schedule: its lattice (-1 ends a
// block's list) and its first logical column and row.
struct alignas(16) TileRec {
    int32_t lat, x0, y0, pad;
};

struct LatState {
    double ledger[4];               // A, B, solute, deposit moved by growth
    unsigned long long closure;     // first closure step count, ~0 if none
    int32_t nonfinite;
    int32_t pad;
};

// Per-column partial results of the observables pass.
struct ColObs {
    double mass_a, mass_b, mass_c, mass_m;     // fluid content (s_t)
    double pend_a, pend_b, pend_c, pend_m;     // nodes turned solid last step
    float phi0, phi1;                           // rho_A - rho_B, centerline
    int32_t h, b, t;                            // aperture, wall thickness
    int32_t wet_lo, wet_hi;                     // A majority at wall nodes
    int32_t fl0, fl1;                           // centerline rows fluid
    int32_t nonfinite;
};

struct StepArgs {
    const LatDesc *desc;
    const int32_t *tile_lat;
    const void *fin;        // post-collision populations of the last step
    void *fout;             // post-collision populations of this step
    const __half *min_;     // FP16 storage: moment planes of fin
    __half *mout;           // FP16 storage: moment planes of fout
    uint8_t *mask;
    double *m;
    int32_t *col_fluid;
    LatState *st;
    int64_t *step;          // completed steps (read at start, bumped at end)
    unsigned int *done;     // blocks finished in this launch
    // test hook of the bounded waits: bytes that block 0 expects on top of
    // its first tile's copies and that no copy delivers (0 normally)
    int32_t stall_tx;
};

constexpr int GHOST = 2;  // ghost rows on each side in y
constexpr int OBS_ROWS = 4;  // warps per block of k_obs_columns (32 columns)

// ---- FP16 storage codec ------------------------------------------------------
// A component's moving populations are kept as FP16 deviations from per-node
// references (FP16, stored once per node, component and weight class), the
// solute likewise; the rest population is kept in FP32:
//   moving i = 1..8:  r_c = FP16(w_c rho~) for the class c of i (w_1 or w_5),
//                     d = 2^10 (f_i - r_c) / w_i,  f_i = r_c + (w_i 2^-10) d
//   solute k = 0..3:  r = FP16(C / 4),  d = 2^12 (g_k - r),  g_k = r + 2^-12 d
//   rest:             f_0 in FP32, taking up the moving values' rounding
// The power-of-two scales are exact; they lift the minority component's
// small deviations out of FP16's subnormal range (|d| stays far below
// 65504).  Reading is one fused multiply-add per value, rounded exactly as
// written here (no contraction into later sums), so all code paths rebuild
// the same FP32 value from the same bits.
constexpr float kDevScale = 1024.0f;
constexpr float kInvDevScale = 1.0f / 1024.0f;
constexpr float kSolScale = 4096.0f;
constexpr float kInvSolScale = 1.0f / 4096.0f;

// Moving population i (1..8) of a D2Q9 component from its deviation and the
// reference of its weight class.
__device__ __forceinline__ float dec_pop(int i, float d, float ref) {
    return __fmaf_rn(d, wq(i) * kInvDevScale, ref);
}
// A solute population from its deviation and reference.
__device__ __forceinline__ float dec_sol(float d, float ref) {
    return __fmaf_rn(d, kInvSolScale, ref);
}

// Encodes the 9 post-collision populations of one component: the moving
// deviations into dq[1..8], the references of the two weight classes into
// h1 (w_1 rho~) and h5 (w_5 rho~), the rest population into `rest`.
// rho~ = f_0 / w_0 (the density times 1 - 3/2 u.u at equilibrium), so every
// deviation is small.  The rest population takes up the quantisation error
// of the eight moving ones -- each error f_i - read-back(f_i) is exact in
// FP32 and tiny, and readers round the read-back exactly as here -- so the
// stored mass is the FP32 mass up to one rounding at f_0's magnitude.
// (Solving the rest population from an FP32 sum of all nine values instead
// biased the mass of long runs by about 1e-8 per step: populations near
// w_i rho share their low-order bits, so the roundings of such sums are not
// unbiased.)
__device__ __forceinline__ void enc9(const float f[Q], __half dq[Q],
                                     __half &h1, __half &h5, float &rest) {
    const float rt = f[0] * (1.0f / wq(0));
    h1 = __float2half_rn(wq(1) * rt);
    h5 = __float2half_rn(wq(5) * rt);
    const float ref1 = __half2float(h1), ref5 = __half2float(h5);
    const float n1 = -ref1 * (kDevScale / wq(1)), n5 = -ref5 * (kDevScale / wq(5));
    float err = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float ref = i < 5 ? ref1 : ref5;
        dq[i] = __float2half_rn(__fmaf_rn(f[i], kDevScale / wq(i), i < 5 ? n1 : n5));
        err += f[i] - dec_pop(i, __half2float(dq[i]), ref);
    }
    rest = f[0] + err;
}

// Encodes the 4 solute populations; returns the reference C~ / 4.
__device__ __forceinline__ __half enc4(const float g[QS], __half dq[QS]) {
    const float c = (g[0] + g[2]) + (g[1] + g[3]);
    const __half ch = __float2half_rn(0.25f * c);
    const float ct = __half2float(ch);
#pragma unroll
    for (int k = 0; k < QS; ++k) dq[k] = __float2half_rn((g[k] - ct) * kSolScale);
    return ch;
}

// Reciprocal: the hardware approximation (PTX rcp.approx.ftz.f32, within
// one ulp) refined by one Newton-Raphson step for f(r) = 1/r - x,
// r1 = r0 + r0 (1 - x r0), with the residual 1 - x r0 formed by one fused
// multiply-add.  The approximation alone is biased enough to double the
// drift of a long run against the FP64 solution.  Callers keep the
// argument above 1e-30.
__device__ __forceinline__ float rcp_nr(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = __fmaf_rn(-x, r, 1.0f);
    return __fmaf_rn(r, e, r);
}

constexpr int XGHOST = 16;  // physical columns before logical column 0

// FP16 storage: the FP32 rest planes of lattice d (A, then B, `plane`
// apart), at its logical node (0, 0), inside the moment block that starts
// 5 planes before them.  Both the block start (a multiple of 9 planes of
// halves) and the 5 reference planes keep them 16-byte aligned.
__device__ __forceinline__ float *rest_planes(__half *mom, const LatDesc &d) {
    const int64_t g = (int64_t)GHOST * d.pitch + XGHOST;
    return reinterpret_cast<float *>(mom + (d.mom_off - g) + NMOM * d.plane) + g;
}
__device__ __forceinline__ const float *rest_planes(const __half *mom,
                                                    const LatDesc &d) {
    return rest_planes(const_cast<__half *>(mom), d);
}

// Calls f(offset) for every periodic image of node (x, y) that lies in the
// ghost band (columns -2 .. nx + 1, rows -2 .. ny + 1, the node itself
// excluded); nodes at least two nodes inside the lattice have none.
template <class F>
__device__ __forceinline__ void for_ghosts(int x, int y, int nx, int ny,
                                           int pitch, int own, F f) {
    if (x >= GHOST && x < nx - GHOST && y >= GHOST && y < ny - GHOST) return;
    for (int ky = -2; ky <= 2; ++ky) {
        const int yi = y + ky * ny;
        if (yi < -GHOST || yi >= ny + GHOST) continue;
        for (int kx = -2; kx <= 2; ++kx) {
            if (kx == 0 && ky == 0) continue;
            const int xi = x + kx * nx;
            if (xi < -GHOST || xi >= nx + GHOST) continue;
            f(own + ky * ny * pitch + kx * nx);
        }
    }
}

// Stores a mask byte of node (x, y) and its ghost images.
__device__ __forceinline__ void mask_store(uint8_t *mask, int own, int x,
                                           int y, int nx, int ny, int pitch,
                                           uint8_t v) {
    mask[own] = v;
    for_ghosts(x, y, nx, ny, pitch, own, [&](int off) { mask[off] = v; });
}

// Periodic index for any offset (lattices smaller than a tile included).
__device__ __forceinline__ int wrapg(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}
// Periodic index for a neighbour offset of at most one.
__device__ __forceinline__ int wrap1(int a, int n) {
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

}  // namespace lbmk
