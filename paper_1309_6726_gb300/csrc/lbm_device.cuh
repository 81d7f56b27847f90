// lbm_device.cuh -- device-side layout and lattice constants of the
// reactive two-component lattice Boltzmann library (sm_103a).
//
// Layout in HBM (one handle, `count` lattices packed back to back):
//   populations: two ping-pong buffers of 32-bit words; in each, lattice l
//     owns consecutive planes of (ny + 4) * pitch words, rows padded to
//     `pitch` (a multiple of 32 words, so every row starts on a 128-byte
//     boundary):
//       FP32 storage: 22 planes (A: 9, B: 9, solute: 4);
//       FP16 storage: 15 planes (see the codec below): 8 planes of half2
//       deviation pairs {A_i, B_i} of the moving populations, 2 planes of
//       half2 solute deviation pairs, 2 planes of half2 linear-reference
//       pairs {v_A, v_B} (x, then y) and 3 FP32 reference planes
//       (rho~_A, rho~_B, C~);
//   every plane (populations, mask) has a two-node ghost band around the
//     lattice -- rows -2, -1, ny, ny + 1 and columns -2, -1, nx, nx + 1 --
//     holding the periodic images of the nodes next to the boundaries; the
//     offsets below point at logical node (0, 0), which sits at physical
//     row 2 and column 16 of the lattice's planes, so node (x, y) is at
//     offset y * pitch + x for -2 <= x < nx + 2, -2 <= y < ny + 2; the
//     nodes next to the boundaries refresh their images whenever they write;
//   mask: one byte per node, read and written in place (see MaskBits);
//   deposit: one double per node;
//   per section column: fluid-node counter (closure), initial wall
//     thickness below and above (observables);
//   per lattice: ledgers, closure step, non-finite flag.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbmk {

constexpr int Q = 9;      // D2Q9 per fluid component
constexpr int QS = 4;     // D2Q4 solute
constexpr int NPOP = 22;  // FP32 storage: 9 + 9 + 4 planes per lattice
// FP16 storage: 15 planes of 32-bit words per lattice (see the codec)
constexpr int NW16 = 15;
constexpr int W16_SOL = 8;   // half2 {C_0, C_1}, then {C_2, C_3}
constexpr int W16_VEL = 10;  // half2 {v_A, v_B} along x, then along y
constexpr int W16_REF = 12;  // FP32 rho~_A, rho~_B, C~

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
    int64_t pop_off;    // first word of plane 0 in a population buffer
    int64_t pad64_;
    int64_t plane;      // (ny + 4) * pitch: rows -2 .. ny + 1
    int64_t col_off;    // first section column in per-column arrays
    float tau_a, tau_b, inv_tau_a, inv_tau_b, inv_tau_d;
    float g_coh, g_ads, k_r, c_in, body_x;
    double m_th;
    int32_t index;      // position of this lattice in the batch
    int32_t bf16;       // 16-bit storage: 1 BF16, 0 FP16 (unused for FP32)
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
    uint8_t *mask;
    double *m;
    int32_t *col_fluid;
    LatState *st;
    int64_t *step;          // completed steps (read at start, bumped at end)
    unsigned int *done;     // blocks finished in this launch
    // test hook of the bounded waits: bytes that block 0 expects on top of
    // its first tile's copies and that no copy delivers (0 normally)
    int32_t stall_tx;
    // per lattice {A, B, solute}: this launch adds the fluid content of
    // every node it updates (zeroed before the launch); null on launches
    // that do not sum
    double *sums;
};

// One node's share of StepArgs::sums: rho_A and rho_B as the collision
// conserves them (its post-collision populations sum to these up to FP32
// rounding) and C after the update and the reaction.
struct NodeTot {
    float a, b, c;
};

// One lattice's input arrays (row-major ny * nx) as the device addresses
// them: pinned or registered host memory (mapped into the device's address
// space), managed or this device's memory.  A null entry: the host copied
// that array into the staging area instead (pageable host memory).
struct InPtrs {
    const float *rho_a, *rho_b, *conc;
    const uint8_t *solid;
};

constexpr int GHOST = 2;  // ghost rows on each side in y
constexpr int OBS_ROWS = 4;  // warps per block of k_obs_columns (32 columns)

// ---- 16-bit storage codec (FP16, or BF16) -------------------------------------
// FP16 storage keeps, per node, the populations in scaled form -- f^_i =
// f_i / w_i for the D2Q9 components (the equilibrium is then
// rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u) with no weight) and g^_k = 4 g_k
// for the solute -- as FP16 deviations from a per-node reference that is
// exact in FP32:
//   A, B:   the reference of direction i is linear in e_i,
//             r_i = rho~ + e_i . v,
//           rho~ the rest population f^_0 (FP32) and v = ((f^_1 - f^_3) /
//           2, (f^_2 - f^_4) / 2) rounded to FP16 (the odd part of the
//           axis populations, 3 rho u at equilibrium) for the component
//           with the larger rest population at the node where |v_x| +
//           |v_y| <= f^_0, for the other one at nodes next to a wall where
//           |v_x| + |v_y| <= 4 f^_0, else v = 0;
//           the moving i = 1..8 are
//           stored as d_i = 2^10 (f^_i - r_i) in FP16, the A and B values
//           of one direction (deviations, and v per axis) packed in one
//           half2 word; read back f^_i = r_i + 2^-10 d_i;
//   solute: reference C~ (the concentration), d_k = 2^10 (g^_k - C~), two
//           directions per half2 word; g^_k = C~ + 2^-10 d_k.
// The fluid deviation is then only the even second-order part 9/2 rho
// (e.u)^2 - 3/2 rho u.u plus the non-equilibrium part, so FP16's 11-bit
// significand applies to a quantity about u times smaller than with the
// rest population alone as reference: in a slow bulk flow (u ~ 1e-3) the
// read-back is as accurate as an FP32 value.  With the rest population
// alone the rounding of the 3 rho e.u part (relative 2^-11 of it, at every
// node and step) slowed a 4096 x 128 capillary's imbibition by a few
// percent against FP32 and the FP64 solution; with the linear reference
// the front agrees with FP32 to 0.01 lattice units after 15000 steps.
// At equilibrium the deviation of direction i is 3 rho s + 9/2 rho s^2
// (s = e_i.u) against the rest population and 9/2 rho s^2 against r_i,
// which is no larger for every i exactly when |s| <= 1/3 for every i,
// i.e. |u_x| + |u_y| <= 1/3 or |v_x| + |v_y| <= rho: the writer takes v
// only there (against f^_0 <= rho, so a little inside it).  Beyond it,
// at strongly forced nodes, the linear reference would enlarge the
// deviation of the directions whose linear and quadratic parts have
// opposite signs.  The minority phase is treated apart: away from walls
// it keeps the rest population alone (with v, its worst per-component
// error over 40 steps of a small preform against the FP64 solution grew
// 2.6 times), while next to a wall, where the adhesion force shifts its
// velocity far beyond the majority's, leaving it on the rest population
// made a 4096 x 128 capillary's front drift ahead of FP32 by 2 lattice
// units late in the run; there it takes v up to four times the bound
// above, which keeps that drift four times smaller and the short-run
// errors within their bounds.  The reader does not need to know which was
// chosen: v = 0 reads back as the rest-only reference.
// Since v is rounded to FP16 before either side uses it, writer and reader
// form the same r_i (the mixed fused multiply-adds below; x term first);
// v's own rounding only moves part of the deviation into d.  The
// power-of-two scale keeps small deviations out of FP16's subnormal range.
//
// Mass: the writer quantises every deviation, then adds the exact
// quantisation error sum_i w_i 2^-10 (d_i - FP16(d_i)) (each term exact in
// FP32, the sum small) to the stored reference.  Since rho~ enters all
// nine read-backs with weights summing to one, and the linear terms cancel
// in the weighted sum (sum_i w_i e_i = 0; each r_i is rounded once per
// axis, and is exact when v's last bit is no finer than rho~'s), the
// stored content of the node equals its FP32 post-collision content up to
// roundings at the reference's magnitude, and the shift moves no momentum.
// The solute does the same with weights 1/4.  Readers round every
// read-back exactly as written here (explicit fused multiply-adds), so
// all code paths rebuild the same FP32 values from the same bits.
//
// BF16 in place of FP16 (LBM_BF16): the same layout, scale and steps with
// an 8-bit significand, so each deviation rounds eight times more
// coarsely; its wider exponent range is not needed here (the scaled
// deviations stay far inside FP16's range).  The mass closure is the
// same; the per-value error grows with the significand.
constexpr float kDevScale = 1024.0f;
constexpr float kInvDevScale = 1.0f / 1024.0f;

__device__ __forceinline__ uint16_t lo16(uint32_t w) { return (uint16_t)(w & 0xFFFFu); }
__device__ __forceinline__ uint16_t hi16(uint32_t w) { return (uint16_t)(w >> 16); }

// ---- packed FP32 pairs ------------------------------------------------------
// The FP16 path carries the two fluid components side by side as
// {A, B} float2 values and does their (identical) arithmetic with the
// paired FP32 instructions of sm_100-family GPUs (one instruction, two
// independent IEEE operations, each rounded as its scalar counterpart).
__device__ __forceinline__ float2 f2s(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b (the product by -1 is exact, so this is the rounded difference)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, f2s(-1.0f), a);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
}

// The two 16-bit formats of the deviations: FP16 (11-bit significand,
// the default) and BF16 (8-bit significand, FP32's exponent range).  Both
// use the same layout, scale and read-back; each provides the packing of
// a pair, the mixed-precision fused multiply-add c + h s (FP32 c, 16-bit h
// and s: the product exact, the sum rounded once -- the mixed-precision
// FMA of sm_100-family GPUs, so no separate conversion of h is needed),
// and the 16-bit constants 2^-10, 1 and -1.
struct F16 {
    static constexpr uint16_t kInvDevScale = 0x1400;  // 2^-10
    static constexpr uint16_t kOne = 0x3C00;
    static constexpr uint16_t kMinusOne = 0xBC00;
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static __device__ __forceinline__ float fma(uint16_t h, uint16_t s, float c) {
        float r;
        asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(r) : "h"(h), "h"(s), "f"(c));
        return r;
    }
};
struct BF16 {
    static constexpr uint16_t kInvDevScale = 0x3A80;  // 2^-10
    static constexpr uint16_t kOne = 0x3F80;
    static constexpr uint16_t kMinusOne = 0xBF80;
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static __device__ __forceinline__ float fma(uint16_t h, uint16_t s, float c) {
        float r;
        asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(r) : "h"(h), "h"(s), "f"(c));
        return r;
    }
};

// Reference r_i = rho~ + e_i . v of direction i (1..8) for one component,
// v's 16-bit values vx, vy: one mixed fused multiply-add per nonzero
// component of e_i, x first.  flip: the direction opp(i) instead (e =
// -e_i; the bounced-back value of a pull, a select when i is a constant).
template <class F>
__device__ __forceinline__ float ref_dir(int i, bool flip, float rho,
                                         uint16_t vx, uint16_t vy) {
    float r = rho;
    if (cx(i) != 0) r = F::fma(vx, (cx(i) > 0) != flip ? F::kOne : F::kMinusOne, r);
    if (cy(i) != 0) r = F::fma(vy, (cy(i) > 0) != flip ? F::kOne : F::kMinusOne, r);
    return r;
}

// The {A, B} values of direction i (opp(i) if flip) from their packed
// deviations w, the source's references {rho~_A, rho~_B} and its
// linear-reference words wx, wy (a word the direction does not use is not
// read): r_i + 2^-10 d, rounded as the writer rounds.
template <class F>
__device__ __forceinline__ float2 dec_pair(int i, bool flip, uint32_t w,
                                           float2 ref, uint32_t wx,
                                           uint32_t wy) {
    return make_float2(
        F::fma(lo16(w), F::kInvDevScale, ref_dir<F>(i, flip, ref.x, lo16(wx), lo16(wy))),
        F::fma(hi16(w), F::kInvDevScale, ref_dir<F>(i, flip, ref.y, hi16(wx), hi16(wy))));
}
// Solute direction k from the word of its pair (k even: low half).
template <class F>
__device__ __forceinline__ float dec_sol16(uint32_t w, int k, float ref) {
    return F::fma((k & 1) ? hi16(w) : lo16(w), F::kInvDevScale, ref);
}

// Encodes the scaled post-collision {A, B} values f[0..8] into the 8
// direction words w[0..7], the linear-reference words wv[0..1] (x, y) and
// the references {rho~_A, rho~_B} (mass-exact, see above).  wall: the node
// has a solid neighbour.
template <class F>
__device__ __forceinline__ float2 enc_ab(const float2 f[Q], uint32_t w[8],
                                         uint32_t wv[2], bool wall) {
    // v for the component with the larger rest population (the majority
    // phase at the node) where |v_x| + |v_y| <= f^_0, for the other one at
    // a wall node where |v_x| + |v_y| <= 4 f^_0, 0 otherwise (see above)
    const float2 vx = mul2(f2s(0.5f), sub2(f[1], f[3]));
    const float2 vy = mul2(f2s(0.5f), sub2(f[2], f[4]));
    const float2 va = make_float2(fabsf(vx.x) + fabsf(vy.x), fabsf(vx.y) + fabsf(vy.y));
    const bool ua = f[0].x >= f[0].y ? va.x <= f[0].x : wall && va.x <= 4.f * f[0].x;
    const bool ub = f[0].y >= f[0].x ? va.y <= f[0].y : wall && va.y <= 4.f * f[0].y;
    wv[0] = F::pack(ua ? vx.x : 0.f, ub ? vx.y : 0.f);
    wv[1] = F::pack(ua ? vy.x : 0.f, ub ? vy.y : 0.f);
    float2 e = f2s(0.f);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float2 r = make_float2(ref_dir<F>(i, false, f[0].x, lo16(wv[0]), lo16(wv[1])),
                                     ref_dir<F>(i, false, f[0].y, hi16(wv[0]), hi16(wv[1])));
        // f^_i - r_i is exact where the two are within a factor of two
        // (everywhere the deviation is small), the scale exact
        const float2 dv = mul2(sub2(f[i], r), f2s(kDevScale));
        const uint32_t h = F::pack(dv.x, dv.y);
        // the quantisation errors dv - round(dv), exact
        const float2 q = make_float2(F::fma(lo16(h), F::kMinusOne, dv.x),
                                     F::fma(hi16(h), F::kMinusOne, dv.y));
        e = fma2(f2s(wq(i)), q, e);
        w[i - 1] = h;
    }
    return fma2(e, f2s(kInvDevScale), f[0]);
}

// Encodes the 4 scaled solute values into two words and the reference.
template <class F>
__device__ __forceinline__ void enc_sol(const float gh[QS], uint32_t &w01,
                                        uint32_t &w23, float &rc) {
    const float c = 0.25f * __fadd_rn(__fadd_rn(gh[0], gh[2]),
                                      __fadd_rn(gh[1], gh[3]));
    const float n = -kDevScale * c;
    float d[QS];
#pragma unroll
    for (int k = 0; k < QS; ++k) d[k] = __fmaf_rn(gh[k], kDevScale, n);
    w01 = F::pack(d[0], d[1]);
    w23 = F::pack(d[2], d[3]);
    // the quantisation errors d_k - round(d_k), exact
    const float e = __fadd_rn(
        __fadd_rn(F::fma(lo16(w01), F::kMinusOne, d[0]),
                  F::fma(hi16(w01), F::kMinusOne, d[1])),
        __fadd_rn(F::fma(lo16(w23), F::kMinusOne, d[2]),
                  F::fma(hi16(w23), F::kMinusOne, d[3])));
    rc = __fmaf_rn(e, 0.25f * kInvDevScale, c);
}

// The 15 stored words of a node from its scaled post-collision values, in
// plane order (8 direction pairs, 2 solute pairs, 2 linear-reference
// pairs, rho~_A, rho~_B, C~).
template <class F>
__device__ __forceinline__ void enc_node16(const float2 f[Q], const float gh[QS],
                                           uint32_t v[NW16], bool wall) {
    float rc;
    const float2 r = enc_ab<F>(f, v, v + W16_VEL, wall);
    enc_sol<F>(gh, v[W16_SOL], v[W16_SOL + 1], rc);
    v[W16_REF] = __float_as_uint(r.x);
    v[W16_REF + 1] = __float_as_uint(r.y);
    v[W16_REF + 2] = __float_as_uint(rc);
}

// Densities {rho_A, rho_B} from the scaled {A, B} populations (the same
// rounding everywhere they are formed: own nodes, ring cells, both
// kernels).
__device__ __forceinline__ float2 dens2(const float2 f[Q]) {
    const float2 s1 = add2(add2(f[1], f[3]), add2(f[2], f[4]));
    const float2 s5 = add2(add2(f[5], f[7]), add2(f[6], f[8]));
    return fma2(f2s(wq(0)), f[0], fma2(f2s(wq(1)), s1, mul2(f2s(wq(5)), s5)));
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
