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
// Store16: population i of a node is kept as the FP16 number
//   d_i = (f_i - w_i * rho~) / w_i,
// with rho~ the node's own (post-collision) component density rounded to
// FP16 and stored once per node in a moment plane; the solute likewise as
// d_j = 4 g_j - C~.  Reading rebuilds f_i = w_i (rho~ + d_i) in FP32.  The
// deviation is small next to rho (it carries velocity and non-equilibrium
// parts only), so FP16's relative precision applies to a quantity ~10-100x
// smaller than f_i itself; the minority component (rho ~ 0.006) keeps the
// same relative accuracy as the majority because rho~ is local.  Writing
// divides by the same FP32 weights the reading multiplies by, so the
// weights' rounding cancels.
// ---------------------------------------------------------------------------

struct Store32 {
    static constexpr bool kHalf = false;
    using T = float;
};
struct Store16 {
    static constexpr bool kHalf = true;
    using T = __half;
};

// D2Q9 BGK relaxation towards the equilibrium of (rho, ux, uy).  The rest
// equilibrium is taken as rho minus the eight moving ones (the same value
// in exact arithmetic): the FP32 weights sum to 1 + 7.45e-9, which would
// otherwise create that much mass at every collision.
__device__ __forceinline__ void bgk9(float f[Q], float rho, float ux,
                                     float uy, float inv_tau) {
    const float uu = ux * ux + uy * uy;
    float moving = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float eu = (float)cx(i) * ux + (float)cy(i) * uy;
        const float feq =
            wq(i) * rho * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
        moving += feq;
        f[i] = f[i] - (f[i] - feq) * inv_tau;
    }
    const float feq0 = rho - moving;
    f[0] = f[0] - (f[0] - feq0) * inv_tau;
}

template <class S>
__device__ __forceinline__ void store9(typename S::T *__restrict__ fout,
                                       __half *__restrict__ mout,
                                       const LatDesc &d, int comp,
                                       int64_t own, const float f[Q]) {
    typename S::T *p = fout + d.pop_off + own;
    if constexpr (!S::kHalf) {
#pragma unroll
        for (int i = 0; i < Q; ++i) p[(comp * Q + i) * d.plane] = f[i];
    } else {
        float r = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) r += f[i];
        const __half rh = __float2half_rn(r);
        const float rt = __half2float(rh);
        mout[d.mom_off + comp * d.plane + own] = rh;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            p[(comp * Q + i) * d.plane] = __float2half_rn(f[i] * (1.0f / wq(i)) - rt);
    }
}

template <class S>
__device__ __forceinline__ void store4(typename S::T *__restrict__ fout,
                                       __half *__restrict__ mout,
                                       const LatDesc &d, int64_t own,
                                       const float g[QS]) {
    typename S::T *p = fout + d.pop_off + own;
    if constexpr (!S::kHalf) {
#pragma unroll
        for (int k = 0; k < QS; ++k) p[(2 * Q + k) * d.plane] = g[k];
    } else {
        const float c = g[0] + g[1] + g[2] + g[3];
        const __half ch = __float2half_rn(c);
        const float ct = __half2float(ch);
        mout[d.mom_off + 2 * d.plane + own] = ch;
#pragma unroll
        for (int k = 0; k < QS; ++k) p[(2 * Q + k) * d.plane] = __float2half_rn(4.0f * g[k] - ct);
    }
}

// Everything after the pull, for a node that is fluid in s_t.
//   fA, fB, g: post-streaming populations of the node (g pulled already);
//   rho_nb(c, i): density of component c at x + e_i (0 if solid in s_t);
//   solid_nb(i): 1 if x + e_i is solid in s_t;  solid4(k) for D2Q4 links.
// Returns true if the node reached the threshold in this step.
template <class S, class RhoNb, class SolidNb, class Solid4>
__device__ __forceinline__ bool fluid_update(
    const StepArgs &a, const LatDesc &d, int l, long long t, int gx,
    int64_t own, float fA[Q], float fB[Q], float g[QS], RhoNb rho_nb,
    SolidNb solid_nb, Solid4 solid4) {
    using T = typename S::T;
    T *__restrict__ fout = static_cast<T *>(a.fout);
    // ---- moments ----------------------------------------------------------
    float rA = 0.f, rB = 0.f, jAx = 0.f, jAy = 0.f, jBx = 0.f, jBy = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rA += fA[i];
        rB += fB[i];
        jAx += (float)cx(i) * fA[i];
        jAy += (float)cy(i) * fA[i];
        jBx += (float)cx(i) * fB[i];
        jBy += (float)cy(i) * fB[i];
    }
    // ---- Martys-Chen forces ----------------------------------------------
    float cAx = 0.f, cAy = 0.f, cBx = 0.f, cBy = 0.f, adx = 0.f, ady = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float rbn = rho_nb(1, i);
        const float ran = rho_nb(0, i);
        const float sn = solid_nb(i) ? 1.f : 0.f;
        cAx += wq(i) * rbn * (float)cx(i);
        cAy += wq(i) * rbn * (float)cy(i);
        cBx += wq(i) * ran * (float)cx(i);
        cBy += wq(i) * ran * (float)cy(i);
        adx += wq(i) * sn * (float)cx(i);
        ady += wq(i) * sn * (float)cy(i);
    }
    // G_ads,A = -g_ads, G_ads,B = +g_ads
    const float FAx = -d.g_coh * rA * cAx + d.g_ads * rA * adx + rA * d.body_x;
    const float FAy = -d.g_coh * rA * cAy + d.g_ads * rA * ady;
    const float FBx = -d.g_coh * rB * cBx - d.g_ads * rB * adx + rB * d.body_x;
    const float FBy = -d.g_coh * rB * cBy - d.g_ads * rB * ady;
    // ---- Shan-Chen shift and BGK -----------------------------------------
    const float den = rA * d.inv_tau_a + rB * d.inv_tau_b;
    const float upx = den > 0.f ? (jAx * d.inv_tau_a + jBx * d.inv_tau_b) / den : 0.f;
    const float upy = den > 0.f ? (jAy * d.inv_tau_a + jBy * d.inv_tau_b) / den : 0.f;
    float uAx = upx, uAy = upy, uBx = upx, uBy = upy;
    if (rA > 1e-12f) { uAx += d.tau_a * FAx / rA; uAy += d.tau_a * FAy / rA; }
    if (rB > 1e-12f) { uBx += d.tau_b * FBx / rB; uBy += d.tau_b * FBy / rB; }
    bgk9(fA, rA, uAx, uAy, d.inv_tau_a);
    bgk9(fB, rB, uBx, uBy, d.inv_tau_b);
    // ---- solute ----------------------------------------------------------
    const float rt = rA + rB;
    const float ux = rt > 0.f ? (jAx + jBx + 0.5f * (FAx + FBx)) / rt : 0.f;
    const float uy = rt > 0.f ? (jAy + jBy + 0.5f * (FAy + FBy)) / rt : 0.f;
    if (d.inlet && gx == 0) {
#pragma unroll
        for (int k = 0; k < QS; ++k)
            g[k] = 0.25f * d.c_in * (1.0f + 2.0f * ((float)sx(k) * ux + (float)sy(k) * uy));
    } else {
        const float c = g[0] + g[1] + g[2] + g[3];
#pragma unroll
        for (int k = 0; k < QS; ++k) {
            const float geq = 0.25f * c * (1.0f + 2.0f * ((float)sx(k) * ux + (float)sy(k) * uy));
            g[k] = g[k] - (g[k] - geq) * d.inv_tau_d;
        }
    }
    // ---- surface reaction, deposit, threshold ----------------------------
    int ns = 0;
#pragma unroll
    for (int k = 0; k < QS; ++k) ns += solid4(k) ? 1 : 0;
    bool flagged = false;
    if (ns > 0 && rA > rB) {
        // fraction of the solute consumed, k_r n_s (capped at all of it);
        // applied as g - g * lost rather than g * (1 - lost) so that
        // rounding 1 - lost does not bias the small consumption
        const float cs = g[0] + g[1] + g[2] + g[3];
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
    store9<S>(fout, a.mout, d, 0, own, fA);
    store9<S>(fout, a.mout, d, 1, own, fB);
    store4<S>(fout, a.mout, d, own, g);
    return flagged;
}

// A node flagged in the previous step: its post-streaming fluid, solute and
// deposit go to the lattice ledger.
__device__ __forceinline__ void retire_node(const StepArgs &a,
                                            const LatDesc &d, int l,
                                            int64_t own, const float fA[Q],
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
