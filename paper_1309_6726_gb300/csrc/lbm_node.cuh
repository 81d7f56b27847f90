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
// Store32: plain FP32 planes.
//
// Store16: FP16 deviations from per-node FP16 references, one per component
// and weight class (enc9 / enc4 and dec_pop / dec_sol in lbm_device.cuh).
// The deviation is small next to rho (it carries velocity and
// non-equilibrium parts only), so FP16's relative precision applies to a
// quantity ~10-100x smaller than f_i itself; the minority component
// (rho ~ 0.006) keeps the same relative accuracy as the majority because the
// references are local.  The FP32 rest population absorbs the rounding of
// the eight moving ones so that each node's stored mass equals its FP32
// mass up to one rounding.
// ---------------------------------------------------------------------------

struct Store32 {
    static constexpr bool kHalf = false;
    using T = float;
};
struct Store16 {
    static constexpr bool kHalf = true;
    using T = __half;
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

// FP16 storage: the 20 FP16 deviations of a node at p[sp16(q) * plane],
// its 5 references at mp[refp(c, i) * plane] and mp[kSolRef * plane] and
// its 2 FP32 rest populations at rp[c * rplane].
__device__ __forceinline__ void store22_f16(__half *__restrict__ p,
                                            __half *__restrict__ mp,
                                            float *__restrict__ rp, int plane,
                                            int rplane, const float fA[Q],
                                            const float fB[Q],
                                            const float g[QS]) {
    __half dq[Q];
    float rest;
    __half h1, h5;
    enc9(fA, dq, h1, h5, rest);
    mp[refp(0, 1) * plane] = h1;
    mp[refp(0, 5) * plane] = h5;
    rp[0] = rest;
#pragma unroll
    for (int i = 1; i < Q; ++i) p[sp16(i) * plane] = dq[i];
    enc9(fB, dq, h1, h5, rest);
    mp[refp(1, 1) * plane] = h1;
    mp[refp(1, 5) * plane] = h5;
    rp[rplane] = rest;
#pragma unroll
    for (int i = 1; i < Q; ++i) p[sp16(Q + i) * plane] = dq[i];
    mp[kSolRef * plane] = enc4(g, dq);
#pragma unroll
    for (int k = 0; k < QS; ++k) p[sp16(2 * Q + k) * plane] = dq[k];
}

// Writes the 22 post-collision values of a node at plane offset `off`.
template <class S>
__device__ __forceinline__ void store_node22(const StepArgs &a,
                                             const LatDesc &d, int off,
                                             const float fA[Q],
                                             const float fB[Q],
                                             const float g[QS]) {
    const int pl = (int)d.plane;
    if constexpr (!S::kHalf) {
        store22_f32(static_cast<float *>(a.fout) + d.pop_off + off, pl, fA, fB, g);
    } else {
        store22_f16(static_cast<__half *>(a.fout) + d.pop_off + off,
                    a.mout + d.mom_off + off, rest_planes(a.mout, d) + off, pl,
                    pl, fA, fB, g);
    }
}

// Writes the 22 post-collision values of the tile node at `o` (planes NT
// apart) -- a shared-memory tile that bulk tensor stores then copy out:
// FP32 [22][NT]; FP16 [20][NT] deviations, om [5][NT] references, orest
// [2][NT] rest populations.
template <class S, int NT>
__device__ __forceinline__ void store_tile22(typename S::T *o, __half *om,
                                             float *orest, const float fA[Q],
                                             const float fB[Q],
                                             const float g[QS]) {
    if constexpr (!S::kHalf)
        store22_f32(o, NT, fA, fB, g);
    else
        store22_f16(o, om, orest, NT, NT, fA, fB, g);
}

// Everything after the pull, for a node that is fluid in s_t.
//   fA, fB, g: post-streaming populations of the node (g pulled already);
//   rhoA_nb / rhoB_nb: densities at x + e_i (index 1..8; 0 if solid in s_t);
//   snb: bit i set if x + e_i is solid in s_t;  ns: solid D2Q4 links.
// put(fA, fB, g) writes the node's own post-collision values; its periodic
// images in the ghost band are written here.
// Returns true if the node reached the threshold in this step.
template <class S, class Put>
__device__ __forceinline__ bool fluid_update(
    const StepArgs &a, const LatDesc &d, int l, long long t, int gx, int gy,
    int own, float fA[Q], float fB[Q], float g[QS], const float rhoA_nb[Q],
    const float rhoB_nb[Q], unsigned snb, int ns, Put put) {
    using T = typename S::T;
    // ---- moments ----------------------------------------------------------
    float rA, jAx, jAy, rB, jBx, jBy;
    moments9(fA, rA, jAx, jAy);
    moments9(fB, rB, jBx, jBy);
    // ---- Martys-Chen forces ----------------------------------------------
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
    const float FAx = rA * (d.g_ads * adx - d.g_coh * cAx + d.body_x);
    const float FAy = rA * (d.g_ads * ady - d.g_coh * cAy);
    const float FBx = rB * (-d.g_ads * adx - d.g_coh * cBx + d.body_x);
    const float FBy = rB * (-d.g_ads * ady - d.g_coh * cBy);
    // ---- Shan-Chen shift and BGK -----------------------------------------
    const float den = rA * d.inv_tau_a + rB * d.inv_tau_b;
    const float iden = den > 1e-30f ? rcp_nr(den) : 0.f;
    const float upx = (jAx * d.inv_tau_a + jBx * d.inv_tau_b) * iden;
    const float upy = (jAy * d.inv_tau_a + jBy * d.inv_tau_b) * iden;
    const float sA = rA > 1e-12f ? d.tau_a * rcp_nr(rA) : 0.f;
    const float sB = rB > 1e-12f ? d.tau_b * rcp_nr(rB) : 0.f;
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
    if (ns > 0 && rA > rB) {
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
    put(fA, fB, g);
    // periodic images in the ghost band
    for_ghosts(gx, gy, d.nx, d.ny, d.pitch, own,
               [&](int off) { store_node22<S>(a, d, off, fA, fB, g); });
    return flagged;
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
