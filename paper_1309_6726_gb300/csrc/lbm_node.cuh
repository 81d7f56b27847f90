// lbm_node.cuh -- the per-node part of the fused step shared by the two
// step kernels (direct loads in lbm_step.cu, TMA-staged tiles in
// lbm_step_tma.cu): given the node's pulled populations, the densities of
// its eight neighbours and the mask bytes around it, do the collision,
// the solute update, the surface reaction, the deposit and threshold test,
// and write the node's post-collision state.
#pragma once

#include "lbm_device.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// Population storage policies.
//
// Store32: plain FP32 planes, collision in the populations themselves.
//
// Store16<F>: 16-bit deviations (F = F16 or BF16) from per-node references
// (FP32 rest population plus a 16-bit linear term), A and B of one
// direction packed in one 32-bit word (enc_node16 / dec_pair in
// lbm_device.cuh); the collision works on the scaled populations f_i / w_i
// and 4 g_k (fluid_update16).
// ---------------------------------------------------------------------------

struct Store32 {
    static constexpr bool kHalf = false;
    using T = float;
    using Fmt = F16;  // unused (no 16-bit values)
    static constexpr int kPlanes = NPOP;
};
template <class F>
struct Store16 {
    static constexpr bool kHalf = true;
    using T = uint32_t;
    using Fmt = F;
    static constexpr int kPlanes = NW16;
};

// D2Q9 BGK relaxation towards the equilibrium of (rho, ux, uy),
//   f_i^eq = w_i rho (1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u.u),
// evaluated pairwise: opposite directions share rho (1 - 3/2 u.u) +
// 9/2 rho (e.u)^2 and differ in the sign of 3 rho e.u.  The rest
// equilibrium is rho minus the eight moving ones (the same value in exact
// arithmetic): the FP32 weights sum to 1 + 7.45e-9, which would otherwise
// create that much mass at every collision.
__device__ __forceinline__ void bgk9(float f[Q], float rho, float ux,
                                     float uy, float omega) {
    const float a = rho * (1.0f - 1.5f * (ux * ux + uy * uy));
    const float r3 = 3.0f * rho, r45 = 4.5f * rho;
    const float up = ux + uy, um = ux - uy;
    const float sx_ = a + r45 * ux * ux, sy_ = a + r45 * uy * uy;
    const float sp = a + r45 * up * up, sm = a + r45 * um * um;
    const float px = r3 * ux, py = r3 * uy, pp = r3 * up, pm = r3 * um;
    const float w1 = wq(1), w5 = wq(5);
    float feq[Q];
    feq[1] = w1 * (sx_ + px);
    feq[3] = w1 * (sx_ - px);
    feq[2] = w1 * (sy_ + py);
    feq[4] = w1 * (sy_ - py);
    feq[5] = w5 * (sp + pp);   // (1, 1)
    feq[7] = w5 * (sp - pp);   // (-1, -1)
    feq[8] = w5 * (sm + pm);   // (1, -1)
    feq[6] = w5 * (sm - pm);   // (-1, 1)
    feq[0] = rho - (((feq[1] + feq[3]) + (feq[2] + feq[4])) +
                    ((feq[5] + feq[7]) + (feq[6] + feq[8])));
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = f[i] + omega * (feq[i] - f[i]);
}

// Density and momentum of 9 populations.
__device__ __forceinline__ void moments9(const float f[Q], float &r,
                                         float &jx, float &jy) {
    r = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) +
        ((f[5] + f[7]) + (f[6] + f[8]));
    jx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
    jy = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
}

// sum_i w_i v(x + e_i) e_i for the eight neighbours v[1..8].
__device__ __forceinline__ void stencil9(const float v[Q], float &sx_,
                                         float &sy_) {
    const float d1 = v[5] - v[7], d2 = v[8] - v[6];  // (1,1)-(-1,-1), (1,-1)-(-1,1)
    sx_ = wq(1) * (v[1] - v[3]) + wq(5) * (d1 + d2);
    sy_ = wq(1) * (v[2] - v[4]) + wq(5) * (d1 - d2);
}

// FP32 storage: the 22 values of a node at p[q * plane].
__device__ __forceinline__ void store22_f32(float *__restrict__ p, int plane,
                                            const float fA[Q],
                                            const float fB[Q],
                                            const float g[QS]) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        p[i * plane] = fA[i];
        p[(Q + i) * plane] = fB[i];
    }
#pragma unroll
    for (int k = 0; k < QS; ++k) p[(2 * Q + k) * plane] = g[k];
}

// FP16 storage: the 15 words of a node at p[w * plane].
__device__ __forceinline__ void store_words16(uint32_t *__restrict__ p,
                                              int plane,
                                              const uint32_t v[NW16]) {
#pragma unroll
    for (int w = 0; w < NW16; ++w) p[w * plane] = v[w];
}

// FP32 storage: writes the 22 post-collision values of a node at plane
// offset `off`.
__device__ __forceinline__ void store_node22(const StepArgs &a,
                                             const LatDesc &d, int off,
                                             const float fA[Q],
                                             const float fB[Q],
                                             const float g[QS]) {
    store22_f32(static_cast<float *>(a.fout) + d.pop_off + off, (int)d.plane,
                fA, fB, g);
}

// Martys-Chen cohesion and adhesion forces and the Shan-Chen velocity
// shift of a fluid node (readings c1, c3, c4):
//   F_s = rho_s (G_ads,s sum_i w_i s(x + e_i) e_i
//                - G_c sum_i w_i rho_s'(x + e_i) e_i + body force),
//   u' = sum_s (j_s / tau_s) / sum_s (rho_s / tau_s),
//   u_s^eq = u' + tau_s F_s / rho_s   (= u' where rho_s < 1e-12).
// The densities and momenta may be in any units whose density is the
// component's mass (the FP16 path passes sums of scaled populations with
// their weights applied).
struct Shift {
    float FAx, FAy, FBx, FBy;  // forces on A and B
    float upx, upy;            // common velocity u'
    float sA, sB;              // tau_s / rho_s
};
__device__ __forceinline__ Shift forces_shift(const LatDesc &d, float rA,
                                              float rB, float jAx, float jAy,
                                              float jBx, float jBy,
                                              const float rhoA_nb[Q],
                                              const float rhoB_nb[Q],
                                              unsigned snb) {
    Shift r;
    float cAx, cAy, cBx, cBy, adx, ady;
    stencil9(rhoB_nb, cAx, cAy);  // A feels B
    stencil9(rhoA_nb, cBx, cBy);  // B feels A
    if (snb == 0u) {  // no solid neighbour (most nodes): the stencil is 0
        adx = 0.f;
        ady = 0.f;
    } else {
        float sv[Q];
#pragma unroll
        for (int i = 1; i < Q; ++i) sv[i] = ((snb >> i) & 1u) ? 1.f : 0.f;
        stencil9(sv, adx, ady);
    }
    // G_ads,A = -g_ads, G_ads,B = +g_ads
    r.FAx = rA * (d.g_ads * adx - d.g_coh * cAx + d.body_x);
    r.FAy = rA * (d.g_ads * ady - d.g_coh * cAy);
    r.FBx = rB * (-d.g_ads * adx - d.g_coh * cBx + d.body_x);
    r.FBy = rB * (-d.g_ads * ady - d.g_coh * cBy);
    const float den = rA * d.inv_tau_a + rB * d.inv_tau_b;
    const float iden = den > 1e-30f ? rcp_nr(den) : 0.f;
    r.upx = (jAx * d.inv_tau_a + jBx * d.inv_tau_b) * iden;
    r.upy = (jAy * d.inv_tau_a + jBy * d.inv_tau_b) * iden;
    r.sA = rA > 1e-12f ? d.tau_a * rcp_nr(rA) : 0.f;
    r.sB = rB > 1e-12f ? d.tau_b * rcp_nr(rB) : 0.f;
    return r;
}

// Everything after the pull, for a node that is fluid in s_t.
//   fA, fB, g: post-streaming populations of the node (g pulled already);
//   rhoA_nb / rhoB_nb: densities at x + e_i (index 1..8; 0 if solid in s_t);
//   snb: bit i set if x + e_i is solid in s_t;  ns: solid D2Q4 links.
// put(fA, fB, g) writes the node's own post-collision values; its periodic
// images in the ghost band are written here.  want: also sets tot to the
// node's fluid content (NodeTot).
// Returns true if the node reached the threshold in this step.
template <class Put>
__device__ __forceinline__ bool fluid_update(
    const StepArgs &a, const LatDesc &d, int l, long long t, int gx, int gy,
    int own, float fA[Q], float fB[Q], float g[QS], const float rhoA_nb[Q],
    const float rhoB_nb[Q], unsigned snb, int ns, Put put, bool want,
    NodeTot &tot) {
    // ---- moments ----------------------------------------------------------
    float rA, jAx, jAy, rB, jBx, jBy;
    moments9(fA, rA, jAx, jAy);
    moments9(fB, rB, jBx, jBy);
    const Shift sh = forces_shift(d, rA, rB, jAx, jAy, jBx, jBy, rhoA_nb,
                                  rhoB_nb, snb);
    const float FAx = sh.FAx, FAy = sh.FAy, FBx = sh.FBx, FBy = sh.FBy;
    const float upx = sh.upx, upy = sh.upy, sA = sh.sA, sB = sh.sB;
    bgk9(fA, rA, upx + sA * FAx, upy + sA * FAy, d.inv_tau_a);
    bgk9(fB, rB, upx + sB * FBx, upy + sB * FBy, d.inv_tau_b);
    // ---- solute ----------------------------------------------------------
    const float rt = rA + rB;
    const float irt = rt > 1e-30f ? rcp_nr(rt) : 0.f;
    const float ux = ((jAx + jBx) + 0.5f * (FAx + FBx)) * irt;
    const float uy = ((jAy + jBy) + 0.5f * (FAy + FBy)) * irt;
    {
        const bool inl = d.inlet && gx == 0;
        const float c = inl ? d.c_in : (g[0] + g[2]) + (g[1] + g[3]);
        const float q = 0.25f * c, hx2 = 0.5f * c * ux, hy2 = 0.5f * c * uy;
        const float geq[QS] = {q + hx2, q + hy2, q - hx2, q - hy2};
        const float om = inl ? 1.0f : d.inv_tau_d;
#pragma unroll
        for (int k = 0; k < QS; ++k) g[k] = g[k] + om * (geq[k] - g[k]);
    }
    // ---- surface reaction, deposit, threshold ----------------------------
    bool flagged = false;
    const bool react = ns > 0 && rA > rB;
    if (react) {
        // fraction of the solute consumed, k_r n_s (capped at all of it);
        // applied as g - g * lost rather than g * (1 - lost) so that
        // rounding 1 - lost does not bias the small consumption
        const float cs = (g[0] + g[2]) + (g[1] + g[3]);
        const float lost = fminf(1.0f, d.k_r * (float)ns);
#pragma unroll
        for (int k = 0; k < QS; ++k) g[k] -= g[k] * lost;
        const double dM = (double)cs * (double)lost;
        double *mp = a.m + d.node_off + own;
        const double mv = *mp + dM;
        *mp = mv;
        if (mv >= d.m_th) {
            flagged = true;
            if (gx >= d.cap_x0 && gx < d.cap_x1) {
                const int old = atomicSub(&a.col_fluid[d.col_off + gx - d.cap_x0], 1);
                if (old == 1) atomicMin(&a.st[l].closure, (unsigned long long)(t + 1));
            }
        }
    }
    if (!(rt < 3.0e38f)) atomicOr(&a.st[l].nonfinite, 1);
    if (want) {
        tot.a = rA;
        tot.b = rB;
        tot.c = (g[0] + g[2]) + (g[1] + g[3]);
    }
    put(fA, fB, g);
    // periodic images in the ghost band
    for_ghosts(gx, gy, d.nx, d.ny, d.pitch, own,
               [&](int off) { store_node22(a, d, off, fA, fB, g); });
    return flagged;
}

// ---------------------------------------------------------------------------
// FP16 storage: the same update on scaled populations f^_i = f_i / w_i and
// g^_k = 4 g_k, the two fluid components side by side as {A, B} pairs
// (packed FP32 instructions, lbm_device.cuh).
// ---------------------------------------------------------------------------

// Momenta {j_A, j_B} from scaled populations, j = sum_i w_i f^_i e_i.
__device__ __forceinline__ void mom2(const float2 f[Q], float2 &jx,
                                     float2 &jy) {
    const float2 d57 = sub2(f[5], f[7]);
    jx = fma2(f2s(wq(1)), sub2(f[1], f[3]),
              mul2(f2s(wq(5)), add2(d57, sub2(f[8], f[6]))));
    jy = fma2(f2s(wq(1)), sub2(f[2], f[4]),
              mul2(f2s(wq(5)), add2(d57, sub2(f[6], f[8]))));
}

// sum_i w_i v(x + e_i) e_i for eight neighbour pairs v[1..8].
__device__ __forceinline__ void stencil2(const float2 v[Q], float2 &sx_,
                                         float2 &sy_) {
    const float2 d1 = sub2(v[5], v[7]), d2 = sub2(v[8], v[6]);
    sx_ = fma2(f2s(wq(1)), sub2(v[1], v[3]), mul2(f2s(wq(5)), add2(d1, d2)));
    sy_ = fma2(f2s(wq(1)), sub2(v[2], v[4]), mul2(f2s(wq(5)), sub2(d1, d2)));
}

// BGK relaxation of scaled {A, B} populations towards
//   f^eq_i = rho (1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u.u),
// pairwise as bgk9.  The rest value closes the mass exactly as dens2 forms
// it: w_0 f^eq_0 = rho - (w_1 S_1 + w_5 S_5), the quotient by the FP32 w_0
// taken as a product with 9/4 and one fused multiply-add correction (9/4
// alone would make w_0 f^eq_0 exceed its target by 7e-9, mass created at
// every collision).
__device__ __forceinline__ void bgk2(float2 f[Q], float2 rho, float2 ux,
                                     float2 uy, float2 omega) {
    const float2 uu = fma2(ux, ux, mul2(uy, uy));
    const float2 a = mul2(rho, fma2(f2s(-1.5f), uu, f2s(1.0f)));
    const float2 r3 = mul2(f2s(3.0f), rho), r45 = mul2(f2s(4.5f), rho);
    const float2 up = add2(ux, uy), um = sub2(ux, uy);
    const float2 sx_ = fma2(mul2(r45, ux), ux, a), sy_ = fma2(mul2(r45, uy), uy, a);
    const float2 sp = fma2(mul2(r45, up), up, a), sm = fma2(mul2(r45, um), um, a);
    const float2 px = mul2(r3, ux), py = mul2(r3, uy);
    const float2 pp = mul2(r3, up), pm = mul2(r3, um);
    float2 feq[Q];
    feq[1] = add2(sx_, px);
    feq[3] = sub2(sx_, px);
    feq[2] = add2(sy_, py);
    feq[4] = sub2(sy_, py);
    feq[5] = add2(sp, pp);   // (1, 1)
    feq[7] = sub2(sp, pp);   // (-1, -1)
    feq[8] = add2(sm, pm);   // (1, -1)
    feq[6] = sub2(sm, pm);   // (-1, 1)
    const float2 s1 = add2(add2(feq[1], feq[3]), add2(feq[2], feq[4]));
    const float2 s5 = add2(add2(feq[5], feq[7]), add2(feq[6], feq[8]));
    const float2 v = sub2(rho, fma2(f2s(wq(1)), s1, mul2(f2s(wq(5)), s5)));
    const float2 y0 = mul2(v, f2s(2.25f));
    feq[0] = fma2(fma2(f2s(-wq(0)), y0, v), f2s(2.25f), y0);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = fma2(omega, sub2(feq[i], f[i]), f[i]);
}

// 1 / x by the hardware approximation and one Newton-Raphson step, for a
// pair, 0 where x <= lim (as rcp_nr).
__device__ __forceinline__ float2 rcp2_guard(float2 x, float lim) {
    float2 r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(x.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(x.y));
    const float2 e = fma2(make_float2(-x.x, -x.y), r, f2s(1.0f));
    r = fma2(r, e, r);
    return make_float2(x.x > lim ? r.x : 0.f, x.y > lim ? r.y : 0.f);
}

// Everything after the pull for a node fluid in s_t, 16-bit storage of
// format F.
//   f, g: scaled post-streaming {A, B} populations and solute of the node;
//   rho: its densities {rho_A, rho_B} (dens2 of f, as in the density frame);
//   nb: densities {rho_A, rho_B} at x + e_i (index 1..8; 0 if solid);
//   snb, ns: as for fluid_update.
// The forces and the shift are those of forces_shift (readings c1, c3, c4),
// formed for both components at once.  put(words) writes the node's 15
// stored words; its periodic images in the ghost band are written here.
// want: also sets tot to the node's fluid content (NodeTot).
// Returns true if the node reached the threshold in this step.
template <class F, class Put>
__device__ __forceinline__ bool fluid_update16(
    const StepArgs &a, const LatDesc &d, int l, long long t, int gx, int gy,
    int own, float2 f[Q], float g[QS], float2 rho, const float2 nb[Q],
    unsigned snb, int ns, Put put, bool want, NodeTot &tot) {
    float2 jx, jy;
    mom2(f, jx, jy);
    // ---- Martys-Chen forces: A feels B, B feels A -------------------------
    float2 sw[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) sw[i] = make_float2(nb[i].y, nb[i].x);
    float2 cx2, cy2;
    stencil2(sw, cx2, cy2);
    float adx = 0.f, ady = 0.f;
    if (snb != 0u) {  // solid neighbours: adhesion stencil
        float sv[Q];
#pragma unroll
        for (int i = 1; i < Q; ++i) sv[i] = ((snb >> i) & 1u) ? 1.f : 0.f;
        stencil9(sv, adx, ady);
    }
    // G_ads,A = -g_ads, G_ads,B = +g_ads
    const float2 gx2 = make_float2(d.g_ads * adx + d.body_x, -d.g_ads * adx + d.body_x);
    const float2 gy2 = make_float2(d.g_ads * ady, -d.g_ads * ady);
    const float2 Fx = mul2(rho, fma2(f2s(-d.g_coh), cx2, gx2));
    const float2 Fy = mul2(rho, fma2(f2s(-d.g_coh), cy2, gy2));
    // ---- Shan-Chen shift and BGK -----------------------------------------
    const float2 itau = make_float2(d.inv_tau_a, d.inv_tau_b);
    const float2 tau = make_float2(d.tau_a, d.tau_b);
    const float2 rw = mul2(rho, itau), jxw = mul2(jx, itau), jyw = mul2(jy, itau);
    const float den = rw.x + rw.y;
    const float iden = den > 1e-30f ? rcp_nr(den) : 0.f;
    const float upx = (jxw.x + jxw.y) * iden, upy = (jyw.x + jyw.y) * iden;
    const float2 sh = mul2(tau, rcp2_guard(rho, 1e-12f));
    bgk2(f, rho, fma2(sh, Fx, f2s(upx)), fma2(sh, Fy, f2s(upy)), itau);
    // ---- solute (scaled: g^eq_k = C (1 + 2 e_k.u), C = sum_k g^_k / 4) --
    const float rt = rho.x + rho.y;
    const float irt = rt > 1e-30f ? rcp_nr(rt) : 0.f;
    const float ux = ((jx.x + jx.y) + 0.5f * (Fx.x + Fx.y)) * irt;
    const float uy = ((jy.x + jy.y) + 0.5f * (Fy.x + Fy.y)) * irt;
    {
        const bool inl = d.inlet && gx == 0;
        const float c = inl ? d.c_in : 0.25f * ((g[0] + g[2]) + (g[1] + g[3]));
        const float hx2 = 2.0f * c * ux, hy2 = 2.0f * c * uy;
        const float geq[QS] = {c + hx2, c + hy2, c - hx2, c - hy2};
        const float om = inl ? 1.0f : d.inv_tau_d;
#pragma unroll
        for (int k = 0; k < QS; ++k) g[k] = g[k] + om * (geq[k] - g[k]);
    }
    // ---- surface reaction, deposit, threshold ----------------------------
    bool flagged = false;
    const bool react = ns > 0 && rho.x > rho.y;
    if (react) {
        const float cs = 0.25f * ((g[0] + g[2]) + (g[1] + g[3]));
        const float lost = fminf(1.0f, d.k_r * (float)ns);
#pragma unroll
        for (int k = 0; k < QS; ++k) g[k] -= g[k] * lost;
        const double dM = (double)cs * (double)lost;
        double *mp = a.m + d.node_off + own;
        const double mv = *mp + dM;
        *mp = mv;
        if (mv >= d.m_th) {
            flagged = true;
            if (gx >= d.cap_x0 && gx < d.cap_x1) {
                const int old = atomicSub(&a.col_fluid[d.col_off + gx - d.cap_x0], 1);
                if (old == 1) atomicMin(&a.st[l].closure, (unsigned long long)(t + 1));
            }
        }
    }
    if (!(rt < 3.0e38f)) atomicOr(&a.st[l].nonfinite, 1);
    uint32_t v[NW16];
    enc_node16<F>(f, g, v, snb != 0u);
    if (want) {
        tot.a = rho.x;
        tot.b = rho.y;
        tot.c = 0.25f * ((g[0] + g[2]) + (g[1] + g[3]));
    }
    put(v);
    // periodic images in the ghost band
    uint32_t *out = static_cast<uint32_t *>(a.fout) + d.pop_off;
    for_ghosts(gx, gy, d.nx, d.ny, d.pitch, own,
               [&](int off) { store_words16(out + off, (int)d.plane, v); });
    return flagged;
}

// FP16 storage: a node flagged in the previous step hands its scaled
// post-streaming content (weights applied) and its deposit to the ledger.
__device__ __forceinline__ void retire_node16(const StepArgs &a,
                                              const LatDesc &d, int l,
                                              int own, const float2 f[Q],
                                              const float g[QS]) {
    double ra = 0, rb = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        ra += (double)wq(i) * f[i].x;
        rb += (double)wq(i) * f[i].y;
    }
    const double c = 0.25 * ((double)g[0] + g[1] + g[2] + g[3]);
    double *mp = a.m + d.node_off + own;
    const double mv = *mp;
    *mp = 0.0;
    atomicAdd(&a.st[l].ledger[0], ra);
    atomicAdd(&a.st[l].ledger[1], rb);
    atomicAdd(&a.st[l].ledger[2], c);
    atomicAdd(&a.st[l].ledger[3], mv);
}

// A node flagged in the previous step: its post-streaming fluid, solute and
// deposit go to the lattice ledger.
__device__ __forceinline__ void retire_node(const StepArgs &a,
                                            const LatDesc &d, int l,
                                            int own, const float fA[Q],
                                            const float fB[Q],
                                            const float g[QS]) {
    double ra = 0, rb = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) { ra += fA[i]; rb += fB[i]; }
    const double c = (double)g[0] + g[1] + g[2] + g[3];
    double *mp = a.m + d.node_off + own;
    const double mv = *mp;
    *mp = 0.0;
    atomicAdd(&a.st[l].ledger[0], ra);
    atomicAdd(&a.st[l].ledger[1], rb);
    atomicAdd(&a.st[l].ledger[2], c);
    atomicAdd(&a.st[l].ledger[3], mv);
}

// Lattice totals of a summing launch.  Each thread keeps running FP32
// totals of its nodes in the consecutive tiles of one lattice, with the
// rounding error of every addition carried along (two-sum); when the block
// moves to another lattice, and at the end of the launch, each warp
// reduces them the same way and lane 0 adds the result to StepArgs::sums
// in FP64.  FP64 arithmetic runs at a small fraction of the FP32 rate on
// this GPU and a warp shuffle takes an issue slot of the whole SM, so
// neither is on the per-node path.

// s + e = a + b exactly (Knuth's two-sum; round-to-nearest FP32).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

struct TotAcc {
    float s[3], e[3];  // A, B, solute: sum and accumulated error
    int l;             // lattice, -1 before the first tile
};

__device__ __forceinline__ void tot_reset(TotAcc &c, int l) {
#pragma unroll
    for (int j = 0; j < 3; ++j) { c.s[j] = 0.f; c.e[j] = 0.f; }
    c.l = l;
}

// Reduces the warp's totals (every lane calls it; after the butterfly all
// lanes hold the same sums) and lane 0 adds them to its lattice's sums.
__device__ __forceinline__ void tot_flush(const TotAcc &c, double *sums,
                                          int lane) {
    if (c.l < 0) return;
    float v[3], e[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) { v[j] = c.s[j]; e[j] = c.e[j]; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float pv = __shfl_xor_sync(0xffffffffu, v[j], o);
            const float pe = __shfl_xor_sync(0xffffffffu, e[j], o);
            float r;
            two_sum(v[j], pv, v[j], r);
            e[j] = __fadd_rn(__fadd_rn(e[j], pe), r);
        }
    if (lane == 0) {
        double *dst = sums + 3 * c.l;
#pragma unroll
        for (int j = 0; j < 3; ++j) atomicAdd(dst + j, (double)v[j] + (double)e[j]);
    }
}

// Adds this thread's node of a tile of lattice l (every lane of the warp
// calls it, with the same l).
__device__ __forceinline__ void tot_add(TotAcc &c, const NodeTot &t, int l,
                                        double *sums, int lane) {
    if (l != c.l) {
        tot_flush(c, sums, lane);
        tot_reset(c, l);
    }
    const float v[3] = {t.a, t.b, t.c};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float r;
        two_sum(c.s[j], v[j], c.s[j], r);
        c.e[j] = __fadd_rn(c.e[j], r);
    }
}

// The last block of a launch to finish advances the step counter for the
// next launch (every block read it before taking its ticket).
__device__ __forceinline__ void finish_launch(const StepArgs &a, long long t) {
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(a.done, 1u);
        if (ticket == gridDim.x - 1) {
            *(volatile long long *)a.step = t + 1;
            *a.done = 0u;
            __threadfence();
        }
    }
}

}  // namespace lbmk
