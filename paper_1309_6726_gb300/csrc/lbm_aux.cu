// lbm_aux.cu -- kernels around the time step: building the stored state
// from post-streaming fields (initial state, user-set fields, loading),
// reading it back as post-streaming fields, and the observables of the
// paper's Sec. III (front, wetted length, radii, Delta e, masses, closure).
//
// The step kernel stores the post-collision populations of the last step
// (pull scheme).  The post-streaming state f(t) the method is stated in is
// therefore one pull away; "unstream" is its exact inverse:
//   f*_i(x) = f_i(x + e_i)        if x + e_i is fluid,
//   f*_i(x) = f_{opp i}(x)        if x + e_i is solid (it bounced back).
#include "lbm_node.cuh"

namespace lbmk {

// Stored value q (0..21: A, B, solute) of node offset e, in the
// populations' own units (16-bit storage: read back and unscaled).
template <class F>
__device__ __forceinline__ float load_pop16(const uint32_t *w, const LatDesc &d,
                                            int q, int64_t e) {
    const float *ref = reinterpret_cast<const float *>(w + W16_REF * d.plane);
    if (q < 2 * Q) {
        const int comp = q < Q ? 0 : 1, i = q - comp * Q;
        const float r = ref[comp * d.plane + e];
        if (i == 0) return wq(0) * r;
        const int sh = comp ? 16 : 0;  // B in the high halves
        const float ri = ref_dir<F>(i, false, r, (uint16_t)(w[W16_VEL * d.plane + e] >> sh),
                                    (uint16_t)(w[(W16_VEL + 1) * d.plane + e] >> sh));
        return wq(i) * F::fma((uint16_t)(w[(i - 1) * d.plane + e] >> sh),
                              F::kInvDevScale, ri);
    }
    const int k = q - 2 * Q;
    return 0.25f * dec_sol16<F>(w[(W16_SOL + (k >> 1)) * d.plane + e], k,
                                ref[2 * d.plane + e]);
}
__device__ __forceinline__ float load_pop(const void *base, const LatDesc &d,
                                          bool half, int q, int64_t e) {
    if (!half) return static_cast<const float *>(base)[d.pop_off + q * d.plane + e];
    const uint32_t *w = static_cast<const uint32_t *>(base) + d.pop_off;
    return d.bf16 ? load_pop16<BF16>(w, d, q, e) : load_pop16<F16>(w, d, q, e);
}

// The 15 stored words of a node from its scaled values, in the lattice's
// 16-bit format, encoded as for a node away from walls (any choice of the
// linear reference reads back; the step's encoder gives wall nodes theirs).
__device__ __forceinline__ void enc_node16_d(const LatDesc &d, const float2 f[Q],
                                             const float gh[QS], uint32_t v[NW16]) {
    if (d.bf16)
        enc_node16<BF16>(f, gh, v, false);
    else
        enc_node16<F16>(f, gh, v, false);
}

// load_pop for one storage known at compile time (0 FP32, 1 FP16, 2 BF16).
template <int ST>
__device__ __forceinline__ float load_pop_st(const void *base, const LatDesc &d,
                                             int q, int64_t e) {
    if constexpr (ST == 0) {
        return static_cast<const float *>(base)[d.pop_off + q * d.plane + e];
    } else {
        const uint32_t *w = static_cast<const uint32_t *>(base) + d.pop_off;
        if constexpr (ST == 2) return load_pop16<BF16>(w, d, q, e);
        else return load_pop16<F16>(w, d, q, e);
    }
}

// Post-streaming populations of node (x, y) at the current step: 22 values
// (A, B, solute), pulled from the stored post-collision state with the
// streaming mask bit.  (One straight-line body per storage, so that the
// loads of all directions can be in flight together.)
template <int ST>
__device__ __forceinline__ void pull_node_st(const void *fin,
                                             const uint8_t *mask,
                                             const LatDesc &d, uint8_t pullbit,
                                             int x, int y, float out[NPOP]) {
    const int nx = d.nx, ny = d.ny;
    const int64_t own = (int64_t)y * d.pitch + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int xs = wrap1(x - cx(i), nx), ys = wrap1(y - cy(i), ny);
        const int64_t src = (int64_t)ys * d.pitch + xs;
        const bool b = i != 0 && (mask[src] & pullbit);
        out[i] = load_pop_st<ST>(fin, d, b ? opp(i) : i, b ? own : src);
        out[Q + i] = load_pop_st<ST>(fin, d, Q + (b ? opp(i) : i), b ? own : src);
    }
#pragma unroll
    for (int k = 0; k < QS; ++k) {
        const int xs = wrap1(x - sx(k), nx), ys = wrap1(y - sy(k), ny);
        const int64_t src = (int64_t)ys * d.pitch + xs;
        const bool b = mask[src] & pullbit;
        out[2 * Q + k] = load_pop_st<ST>(fin, d, 2 * Q + (b ? sopp(k) : k), b ? own : src);
    }
}
__device__ __forceinline__ void pull_node(const void *fin,
                                          const uint8_t *mask,
                                          const LatDesc &d, bool half,
                                          uint8_t pullbit, int x, int y,
                                          float out[NPOP]) {
    if (!half)
        pull_node_st<0>(fin, mask, d, pullbit, x, y, out);
    else if (d.bf16)
        pull_node_st<2>(fin, mask, d, pullbit, x, y, out);
    else
        pull_node_st<1>(fin, mask, d, pullbit, x, y, out);
}

// Writes the stored form of node (x, y) from its 22 post-collision values
// (FP16 storage: scaled by 1 / w_i and 4 -- correctly rounded quotients --
// and encoded).
__device__ __forceinline__ void store_node(void *fout, const LatDesc &d,
                                           bool half, int64_t own,
                                           const float v[NPOP]) {
    const int pl = (int)d.plane;
    if (!half) {
        store22_f32(static_cast<float *>(fout) + d.pop_off + own, pl, v, v + Q,
                    v + 2 * Q);
        return;
    }
    float2 f[Q];
    float gh[QS];
    for (int i = 0; i < Q; ++i)
        f[i] = make_float2(__fdiv_rn(v[i], wq(i)), __fdiv_rn(v[Q + i], wq(i)));
    for (int k = 0; k < QS; ++k) gh[k] = 4.0f * v[2 * Q + k];
    uint32_t wv[NW16];
    enc_node16_d(d, f, gh, wv);
    store_words16(static_cast<uint32_t *>(fout) + d.pop_off + own, pl, wv);
}

// ---- set-up of a whole batch, one launch per kernel ------------------------
// The inputs of every lattice sit back to back in device staging: lattice
// l's nodes from in_off[l] (row-major ny*nx), solid bytes in `solid`, the
// densities and concentration in rho3 as [rho_A | rho_B | C] blocks of
// 3 * nx * ny floats from 3 * in_off[l].  One block takes one row of one
// lattice (rows of all lattices numbered through an exclusive prefix of
// per-lattice row counts, count + 1 entries; the block finds its lattice by
// a binary search) and its threads walk the row's columns.

__device__ __forceinline__ int lattice_of(const int64_t *pre, int count,
                                          int64_t g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Copies n values from src (readable by the device) to dst, 16 bytes per
// read where src is 16-byte aligned (the reads cross the host link; the
// device-side writes stay element-wise, dst having no such alignment),
// element by element otherwise and for the tail; the block's threads
// stride over [i0, n) with step `step` in units of 16-byte groups.
template <class T>
__device__ __forceinline__ void gather_array(const T *src, T *dst, int64_t n,
                                             int64_t i0, int64_t step) {
    constexpr int V = 16 / sizeof(T);  // values per 16-byte read
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int64_t nv = n / V;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        for (int64_t q = i0; q < nv; q += step) {
            const uint4 v = s4[q];
            const T *t = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int j = 0; j < V; ++j) dst[q * V + j] = t[j];
        }
        done = nv * V;
    }
    for (int64_t k = done + i0; k < n; k += step) dst[k] = src[k];
}

// Gathers the inputs of lattices [l0, l0 + gridDim.y) into the device
// staging area in one launch, reading the caller's arrays where the device
// can address them (blockIdx.y: the lattice; the blocks in x stride over
// its nodes): rho3 holds [rho_a | rho_b | conc] from 3 * in_off[l], sol the
// solid bytes from in_off[l].  Entries left null were copied by the host.
__global__ void k_gather_inputs(const InPtrs *ptr, int l0,
                                const int64_t *in_off, float *rho3,
                                uint8_t *sol) {
    const int l = l0 + (int)blockIdx.y;
    const InPtrs p = ptr[l];
    const int64_t o = in_off[l], n = in_off[l + 1] - o;
    float *r = rho3 + 3 * o;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (p.rho_a) gather_array(p.rho_a, r, n, i0, step);
    if (p.rho_b) gather_array(p.rho_b, r + n, n, i0, step);
    if (p.conc) gather_array(p.conc, r + 2 * n, n, i0, step);
    if (p.solid) gather_array(p.solid, sol + o, n, i0, step);
}

// Mask bytes over every lattice's ghost band (columns -2 .. nx + 1, rows
// -2 .. ny + 1; every image is its periodic source node): solid -> all
// three time bits set.  grow: prefix of ny + 4 (rows with the band).
__global__ void k_mask_init_all(const LatDesc *desc, int count,
                                const int64_t *grow, const int64_t *in_off,
                                const uint8_t *solid, uint8_t *mask_all) {
    const int l = lattice_of(grow, count, blockIdx.x);
    const LatDesc &d = desc[l];
    const int y = (int)(blockIdx.x - grow[l]) - GHOST;
    const int ys = wrapg(y, d.ny);
    const uint8_t *srow = solid + in_off[l] + (int64_t)ys * d.nx;
    uint8_t *mrow = mask_all + d.node_off + (int64_t)y * d.pitch;
    for (int x = (int)threadIdx.x - GHOST; x < d.nx + GHOST; x += blockDim.x)
        mrow[x] = srow[x >= 0 && x < d.nx ? x : wrapg(x, d.nx)] ? 7 : 0;
}

// Per section column of every lattice: fluid nodes, and the initial wall
// thickness from below and from above (runs of solid from each edge); a
// column solid from the start sets its lattice's closure step to 0.
// cpre: prefix of the section widths (the lattices' col_off).
__global__ void k_col_init_all(const LatDesc *desc, int count,
                               const int64_t *cpre, const int64_t *in_off,
                               const uint8_t *solid, int32_t *col_fluid,
                               int16_t *wall0, LatState *st) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= cpre[count]) return;
    const int l = lattice_of(cpre, count, g);
    const LatDesc &d = desc[l];
    const int x = d.cap_x0 + (int)(g - cpre[l]);
    const uint8_t *sl = solid + in_off[l];
    int fl = 0, b = 0, t = 0;
    bool below = true;
    for (int y = 0; y < d.ny; ++y) {
        const bool sv = sl[(int64_t)y * d.nx + x] != 0;
        fl += !sv;
        if (below && sv) ++b;
        if (!sv) below = false;
        t = sv ? t + 1 : 0;
    }
    if (fl == 0) {
        t = d.ny;  // a fully solid column: both runs are the column
        atomicMin(&st[l].closure, 0ull);  // closed from the start: step 0
    }
    const int64_t k = d.col_off + (x - d.cap_x0);
    col_fluid[k] = fl;
    wall0[2 * k] = (int16_t)min(b, 32767);
    wall0[2 * k + 1] = (int16_t)min(t, 32767);
}

// Stored initial state of every lattice: each fluid node at rest
// equilibrium, f_i = w_i rho, g_k = C / 4 (reading c13), written in the
// pull scheme's stored form (the post-collision values that one pull turns
// into that state: f*_i(x) = f_i(x + e_i), or f_opp i(x) where x + e_i is
// solid).  The mask must be built (k_mask_init_all) first.  rows: prefix
// of ny.
__global__ void k_init_rest_all(const LatDesc *desc, int count,
                                const int64_t *rows, const int64_t *in_off,
                                const float *rho3, const uint8_t *mask_all,
                                void *fout, bool half) {
    const int l = lattice_of(rows, count, blockIdx.x);
    const LatDesc &d = desc[l];
    const int y = (int)(blockIdx.x - rows[l]);
    const uint8_t *mask = mask_all + d.node_off;
    const int64_t N = (int64_t)d.nx * d.ny;
    const float *ra = rho3 + 3 * in_off[l], *rb = ra + N, *cc = ra + 2 * N;
    for (int x = threadIdx.x; x < d.nx; x += blockDim.x) {
        const int64_t own = (int64_t)y * d.pitch + x;
        if (mask[own] & 1) continue;  // solid: never read
        const int64_t r = (int64_t)y * d.nx + x;
        int64_t src[Q], ssrc[QS];
        for (int i = 0; i < Q; ++i) {
            const int xd = wrap1(x + cx(i), d.nx), yd = wrap1(y + cy(i), d.ny);
            const bool b = mask[(int64_t)yd * d.pitch + xd] & 1;
            src[i] = b ? r : (int64_t)yd * d.nx + xd;
        }
        for (int k = 0; k < QS; ++k) ssrc[k] = src[k + 1];  // D2Q4 k = D2Q9 k + 1
        if (half) {
            // the scaled populations f_i / w_i of a node at rest are its
            // density, 4 g_k its concentration: no weights to divide out
            float2 f[Q];
            float gv[QS];
            for (int i = 0; i < Q; ++i) f[i] = make_float2(ra[src[i]], rb[src[i]]);
            for (int k = 0; k < QS; ++k) gv[k] = cc[ssrc[k]];
            uint32_t wv[NW16];
            enc_node16_d(d, f, gv, wv);
            uint32_t *out = static_cast<uint32_t *>(fout) + d.pop_off;
            store_words16(out + own, (int)d.plane, wv);
            for_ghosts(x, y, d.nx, d.ny, d.pitch, (int)own,
                       [&](int off) { store_words16(out + off, (int)d.plane, wv); });
        } else {
            float v[NPOP];
            for (int i = 0; i < Q; ++i) {
                // opposite directions share a weight
                v[i] = wq(i) * ra[src[i]];
                v[Q + i] = wq(i) * rb[src[i]];
            }
            for (int k = 0; k < QS; ++k) v[2 * Q + k] = 0.25f * cc[ssrc[k]];
            store_node(fout, d, half, own, v);
            for_ghosts(x, y, d.nx, d.ny, d.pitch, (int)own,
                       [&](int off) { store_node(fout, d, half, off, v); });
        }
    }
}

// Solid mask of lattice l at the current step (force bit), row-major
// [ny][nx] bytes 0/1.
__global__ void k_solid_mask(const LatDesc *desc, int l,
                             const uint8_t *mask_all, uint8_t force,
                             uint8_t *out) {
    const LatDesc d = desc[l];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= d.nx) return;
    out[(int64_t)y * d.nx + x] =
        (mask_all[d.node_off + (int64_t)y * d.pitch + x] & force) ? 1 : 0;
}

// Solid masks of every lattice at the current step (force bit), each
// row-major [ny][nx] bytes 0/1, back to back in lattice order (in_off: node
// prefix, rows: row prefix).
__global__ void k_solid_mask_all(const LatDesc *desc, int count,
                                 const int64_t *rows, const int64_t *in_off,
                                 const uint8_t *mask_all, uint8_t force,
                                 uint8_t *out) {
    const int l = lattice_of(rows, count, blockIdx.x);
    const LatDesc &d = desc[l];
    const int y = (int)(blockIdx.x - rows[l]);
    const uint8_t *mrow = mask_all + d.node_off + (int64_t)y * d.pitch;
    uint8_t *orow = out + in_off[l] + (int64_t)y * d.nx;
    for (int x = threadIdx.x; x < d.nx; x += blockDim.x)
        orow[x] = (mrow[x] & force) ? 1 : 0;
}

// Stored state from post-streaming fields (exact inverse of the pull).
// The mask must hold no pending flip (force bit == streaming bit).
__global__ void k_unstream(const LatDesc *desc, int l, const float *canon,
                           const uint8_t *mask_all, uint8_t forcebit,
                           void *fout, bool half) {
    const LatDesc d = desc[l];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= d.nx || y >= d.ny) return;
    const uint8_t *mask = mask_all + d.node_off;
    const int64_t own = (int64_t)y * d.pitch + x;
    if (mask[own] & forcebit) return;
    const int64_t P = (int64_t)d.nx * d.ny;
    float v[NPOP];
    for (int i = 0; i < Q; ++i) {
        const int xd = wrap1(x + cx(i), d.nx), yd = wrap1(y + cy(i), d.ny);
        const bool b = mask[(int64_t)yd * d.pitch + xd] & forcebit;
        const int64_t src = b ? (int64_t)y * d.nx + x : (int64_t)yd * d.nx + xd;
        const int qi = b ? opp(i) : i;
        v[i] = canon[qi * P + src];
        v[Q + i] = canon[(Q + qi) * P + src];
    }
    for (int k = 0; k < QS; ++k) {
        const int xd = wrap1(x + sx(k), d.nx), yd = wrap1(y + sy(k), d.ny);
        const bool b = mask[(int64_t)yd * d.pitch + xd] & forcebit;
        const int64_t src = b ? (int64_t)y * d.nx + x : (int64_t)yd * d.nx + xd;
        v[2 * Q + k] = canon[(2 * Q + (b ? sopp(k) : k)) * P + src];
    }
    store_node(fout, d, half, own, v);
    for_ghosts(x, y, d.nx, d.ny, d.pitch, (int)own,
               [&](int off) { store_node(fout, d, half, off, v); });
}

// Post-streaming fields of lattice l at step t into canon ([22][ny][nx]);
// dens ([3][ny][nx]: rho_A, rho_B, C) and dep ([ny][nx]) when not NULL.
// Nodes solid in s_t (including those turned solid last step) read zero.
__global__ void k_export(const LatDesc *desc, int l, const void *fin,
                         const uint8_t *mask_all,
                         const double *m_all, long long t, bool half,
                         float *canon, float *dens, double *dep) {
    const LatDesc d = desc[l];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= d.nx || y >= d.ny) return;
    const MaskBits mb(t);
    const uint8_t *mask = mask_all + d.node_off;
    const int64_t own = (int64_t)y * d.pitch + x;
    const int64_t n = (int64_t)y * d.nx + x;
    const int64_t P = (int64_t)d.nx * d.ny;
    const bool solid = mask[own] & mb.force;
    float v[NPOP];
    if (solid) {
        for (int q = 0; q < NPOP; ++q) v[q] = 0.f;
    } else {
        pull_node(fin, mask, d, half, mb.pull, x, y, v);
    }
    if (canon)
        for (int q = 0; q < NPOP; ++q) canon[q * P + n] = v[q];
    if (dens) {
        float ra = 0.f, rb = 0.f;
        for (int i = 0; i < Q; ++i) { ra += v[i]; rb += v[Q + i]; }
        dens[n] = ra;
        dens[P + n] = rb;
        dens[2 * P + n] = v[18] + v[19] + v[20] + v[21];
    }
    if (dep) dep[n] = solid ? 0.0 : m_all[d.node_off + own];
}

// Folds nodes turned solid in the last step into the ledger now and makes
// the three mask bits agree (used before replacing fields, so that the
// stored state has no pending flip).
__global__ void k_settle(const LatDesc *desc, int l, const void *fin,
                         uint8_t *mask_all, double *m_all,
                         LatState *st, long long t, bool half) {
    const LatDesc d = desc[l];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= d.nx || y >= d.ny) return;
    const MaskBits mb(t);
    uint8_t *mask = mask_all + d.node_off;
    const int64_t own = (int64_t)y * d.pitch + x;
    const uint8_t s = mask[own];
    if ((s & mb.force) && !(s & mb.pull)) {
        float v[NPOP];
        pull_node(fin, mask, d, half, mb.pull, x, y, v);
        double ra = 0, rb = 0;
        for (int i = 0; i < Q; ++i) { ra += v[i]; rb += v[Q + i]; }
        const double c = (double)v[18] + v[19] + v[20] + v[21];
        double *mp = m_all + d.node_off + own;
        atomicAdd(&st[l].ledger[0], ra);
        atomicAdd(&st[l].ledger[1], rb);
        atomicAdd(&st[l].ledger[2], c);
        atomicAdd(&st[l].ledger[3], *mp);
        *mp = 0.0;
    }
}

__global__ void k_mask_agree(const LatDesc *desc, int l, uint8_t *mask_all,
                             long long t) {
    const LatDesc d = desc[l];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= d.nx || y >= d.ny) return;
    const MaskBits mb(t);
    uint8_t *mask = mask_all + d.node_off;
    const int64_t own = (int64_t)y * d.pitch + x;
    mask_store(mask, (int)own, x, y, d.nx, d.ny, d.pitch, (mask[own] & mb.force) ? 7 : 0);
}

// ---------------------------------------------------------------------------
// Observables.  Pass 1: blocks of 32 x OBS_ROWS threads take 32 consecutive
// columns of all lattices (numbered through col_base): lane = column, so
// loads coalesce along rows, and the warps split the rows of each column.
//
// Masses need no pull: streaming with bounce-back hands every stored value
// of a node that was fluid in the last step to exactly one node that was
// fluid then, so the stored values of those nodes sum to the post-streaming
// content of the fluid nodes plus that of the nodes turned solid at the end
// of the last step (the pending ones, pulled separately, which go to the
// ledger).  Only the nodes whose phase the observables need -- the lowest
// and highest fluid row of a column, and the centreline rows -- are pulled,
// once the partial results have met in shared memory.
// Pass 2: one block per lattice reduces the columns.
// ---------------------------------------------------------------------------

struct ObsPart {
    double stored[3], pend[4], dep;
    int h, nonfin, lo, hi;
};

template <class F>
__device__ __forceinline__ void stored_sums16(const void *fin,
                                              const LatDesc &d, int64_t own,
                                              float &sa, float &sb, float &sc) {
    const uint32_t *w = static_cast<const uint32_t *>(fin) + d.pop_off;
    const float *ref = reinterpret_cast<const float *>(w + W16_REF * d.plane);
    const float2 r = make_float2(ref[own], ref[d.plane + own]);
    sa = wq(0) * r.x;
    sb = wq(0) * r.y;
    const uint32_t wx = w[W16_VEL * d.plane + own];
    const uint32_t wy = w[(W16_VEL + 1) * d.plane + own];
    for (int i = 1; i < Q; ++i) {
        const float2 f = dec_pair<F>(i, false, w[(i - 1) * d.plane + own], r, wx, wy);
        sa += wq(i) * f.x;
        sb += wq(i) * f.y;
    }
    const float rc = ref[2 * d.plane + own];
    const uint32_t w01 = w[W16_SOL * d.plane + own];
    const uint32_t w23 = w[(W16_SOL + 1) * d.plane + own];
    sc = 0.f;
    for (int k = 0; k < QS; ++k)
        sc += 0.25f * dec_sol16<F>(k < 2 ? w01 : w23, k, rc);
}
// Sum of the 22 stored values of a node (A, B, solute), as readers decode
// them (the values load_pop returns, summed in the same order; FP16
// storage reads each packed word and each reference once).
__device__ __forceinline__ void stored_sums(const void *fin,
                                            const LatDesc &d, bool half,
                                            int64_t own, float &sa, float &sb,
                                            float &sc) {
    sa = 0.f;
    sb = 0.f;
    sc = 0.f;
    if (half) {
        if (d.bf16)
            stored_sums16<BF16>(fin, d, own, sa, sb, sc);
        else
            stored_sums16<F16>(fin, d, own, sa, sb, sc);
        return;
    }
    for (int i = 0; i < Q; ++i) {
        sa += load_pop(fin, d, half, i, own);
        sb += load_pop(fin, d, half, Q + i, own);
    }
    for (int k = 0; k < QS; ++k) sc += load_pop(fin, d, half, 2 * Q + k, own);
}

// SUMMED: the last step launch added up the fluid content of the nodes it
// updated (StepArgs::sums); the pass then reads the populations only of the
// nodes that turned solid and of the phase rows.
// ST: the storage (0 FP32, 1 FP16, 2 BF16).
template <bool SUMMED, int ST>
__global__ void __launch_bounds__(32 * OBS_ROWS, SUMMED ? 6 : 1)
    k_obs_columns(const LatDesc *desc, const int32_t *col_lat,
                  const int64_t *col_base, int ncols_total, const void *fin,
                  const uint8_t *mask_all,
                  const double *m_all, long long t, ColObs *out) {
    constexpr bool half = ST != 0;
    __shared__ ObsPart part[OBS_ROWS][32];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int c = blockIdx.x * 32 + lane;
    const MaskBits mb(t);
    ObsPart p = {};
    p.lo = 0x7fffffff;  // lowest / highest fluid row of the column
    p.hi = -1;
    if (c < ncols_total) {
        const int l = col_lat[c];
        const LatDesc d = desc[l];
        const int x = (int)(c - col_base[l]);
        const uint8_t *mask = mask_all + d.node_off;
        const double *mcol = m_all + d.node_off;
        // mask statistics, deposit and (unless summed) stored content, row
        // by row; the rows' loads are independent (the deposit is read
        // whatever the node), so the unrolled loop keeps several in flight
        bool pending = false;
#pragma unroll 8
        for (int y = w; y < d.ny; y += OBS_ROWS) {
            const int64_t own = (int64_t)y * d.pitch + x;
            const uint8_t sv = mask[own];
            const double mv = mcol[own];
            const bool fluid_before = !(sv & mb.pull);
            if (!SUMMED && fluid_before) {
                float sa, sb, sc;
                stored_sums(fin, d, half, own, sa, sb, sc);
                if (!(sa + sb < 3.0e38f)) p.nonfin = 1;
                p.stored[0] += sa;
                p.stored[1] += sb;
                p.stored[2] += sc;
            }
            if (sv & mb.force) {
                pending |= fluid_before;
                continue;
            }
            // (FP64 adds are slow on this GPU; most deposits are 0)
            if (__double_as_longlong(mv) != 0) p.dep += mv;
            p.h += 1;
            p.lo = min(p.lo, y);
            p.hi = max(p.hi, y);
        }
        // nodes that turned solid at the end of the last step (few): the
        // content they received and their deposit
        if (pending) {
            float v[NPOP];
            for (int y = w; y < d.ny; y += OBS_ROWS) {
                const int64_t own = (int64_t)y * d.pitch + x;
                const uint8_t sv = mask[own];
                if (!(sv & mb.force) || (sv & mb.pull)) continue;
                pull_node_st<ST>(fin, mask, d, mb.pull, x, y, v);
                double ra = 0, rb = 0;
                for (int i = 0; i < Q; ++i) { ra += v[i]; rb += v[Q + i]; }
                p.pend[0] += ra;
                p.pend[1] += rb;
                p.pend[2] += (double)v[18] + v[19] + v[20] + v[21];
                p.pend[3] += mcol[own];
            }
        }
    }
    part[w][lane] = p;
    __syncthreads();
    // the lowest and highest fluid rows of the column (every warp)
    int lo = 0x7fffffff, hi = -1, hsum = 0;
    for (int k = 0; k < OBS_ROWS; ++k) {
        lo = min(lo, part[k][lane].lo);
        hi = max(hi, part[k][lane].hi);
        hsum += part[k][lane].h;
    }
    // rho_A - rho_B at the rows the observables read, one row per warp (in
    // parallel): the lowest and highest fluid row (wetting phase at the
    // walls) and the two centerline rows
    __shared__ float sphi[4][32];
    __shared__ int sfl[4][32];
    static_assert(OBS_ROWS >= 4, "one warp per phase row");
    int l = 0, ny = 0, x = 0;
    const uint8_t *mask = nullptr;
    LatDesc d;
    if (c < ncols_total) {
        l = col_lat[c];
        d = desc[l];
        x = (int)(c - col_base[l]);
        mask = mask_all + d.node_off;
        ny = d.ny;
    }
    if (w < 4 && c < ncols_total) {
        const int yc0 = (ny - 1) / 2, yc1 = ny / 2;
        const int y = w == 0 ? lo : w == 1 ? hi : w == 2 ? yc0 : yc1;
        // lo/hi rows only where the column has fluid; centerline rows only
        // where fluid now
        bool need = w < 2 ? hsum > 0
                          : !(mask[(int64_t)y * d.pitch + x] & mb.force);
        float ph = 0.f;
        if (need) {
            float v[NPOP];
            pull_node_st<ST>(fin, mask, d, mb.pull, x, y, v);
            float ra = 0.f, rb = 0.f;
            for (int i = 0; i < Q; ++i) { ra += v[i]; rb += v[Q + i]; }
            ph = ra - rb;
        }
        sphi[w][lane] = ph;
        sfl[w][lane] = need;
    }
    __syncthreads();
    if (w != 0 || c >= ncols_total) return;
    double st[3] = {0, 0, 0};
    ColObs o = {};
    for (int k = 0; k < OBS_ROWS; ++k) {  // fixed order
        const ObsPart &q = part[k][lane];
        for (int j = 0; j < 3; ++j) st[j] += q.stored[j];
        o.pend_a += q.pend[0];
        o.pend_b += q.pend[1];
        o.pend_c += q.pend[2];
        o.pend_m += q.pend[3];
        o.mass_m += q.dep;
        o.h += q.h;
        o.nonfinite |= q.nonfin;
    }
    // fluid content: stored content of the nodes fluid in the last step,
    // less what the pending ones received (totals over a lattice are exact;
    // a single column's share is not, streaming crosses columns)
    o.mass_a = st[0] - o.pend_a;
    o.mass_b = st[1] - o.pend_b;
    o.mass_c = st[2] - o.pend_c;
    if (o.h == 0) {
        o.b = ny;
        o.t = ny;
        o.wet_lo = o.wet_hi = 0;
    } else {
        // the walls are the solid runs below the lowest and above the
        // highest fluid row; the wetting phase is read at those rows
        o.b = lo;
        o.t = ny - 1 - hi;
        o.wet_lo = sphi[0][lane] > 0.f;
        o.wet_hi = sphi[1][lane] > 0.f;
    }
    if (sfl[2][lane]) { o.phi0 = sphi[2][lane]; o.fl0 = 1; }
    if (sfl[3][lane]) { o.phi1 = sphi[3][lane]; o.fl1 = 1; }
    out[c] = o;
}

// The column pass for a handle's storage and summing state.
void launch_obs_columns(bool summed, int store, int nb, int ncols,
                        const LatDesc *desc, const int32_t *col_lat,
                        const int64_t *col_base, const void *fin,
                        const uint8_t *mask, const double *m, long long t,
                        ColObs *out, cudaStream_t s) {
    const dim3 blk(32, OBS_ROWS);
#define LBM_OBS(SUM, ST)                                                       \
    k_obs_columns<SUM, ST><<<nb, blk, 0, s>>>(desc, col_lat, col_base, ncols, \
                                              fin, mask, m, t, out)
    if (summed) {
        if (store == 2) LBM_OBS(true, 2);
        else if (store == 1) LBM_OBS(true, 1);
        else LBM_OBS(true, 0);
    } else {
        if (store == 2) LBM_OBS(false, 2);
        else if (store == 1) LBM_OBS(false, 1);
        else LBM_OBS(false, 0);
    }
#undef LBM_OBS
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] += sh[tid + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

struct LbmObsDev {  // mirrors lbm_obs of the public header
    long long step;
    double front, wetted_lower, wetted_upper, r_min, r_h, r_ave, delta_e;
    double precip_mass, mass_a, mass_b, mass_c;
    double ledger_a, ledger_b, ledger_c, ledger_m;
    int closed, nonfinite;
    long long closure_step;
};

// blockDim.x must be 256.
// sums: per lattice {A, B, solute} summed by the last step launch over the
// nodes it updated (null: the column pass summed the stored state).
__global__ void k_obs_reduce(const LatDesc *desc, const int64_t *col_base,
                             const ColObs *cols, const int16_t *wall0,
                             const LatState *st, const double *sums,
                             long long t, LbmObsDev *out) {
    __shared__ double sh[256];
    __shared__ int s_first[2];
    __shared__ int s_min_h;
    const int l = blockIdx.x;
    const LatDesc d = desc[l];
    const ColObs *c = cols + col_base[l];
    const int tid = threadIdx.x;
    const int nx = d.nx, ny = d.ny;
    const int x0 = d.cap_x0, x1 = d.cap_x1, ncap = x1 - x0;
    const int16_t *w0 = wall0 + 2 * d.col_off;  // (b0, t0) per section column
    if (tid == 0) { s_first[0] = s_first[1] = 0x7fffffff; s_min_h = 0x7fffffff; }
    __syncthreads();
    double ma = 0, mb = 0, mc = 0, mm = 0, pa = 0, pb = 0, pc = 0, pm = 0;
    int nonfin = 0;
    for (int x = tid; x < nx; x += blockDim.x) {
        const ColObs &o = c[x];
        ma += o.mass_a; mb += o.mass_b; mc += o.mass_c; mm += o.mass_m;
        pa += o.pend_a; pb += o.pend_b; pc += o.pend_c; pm += o.pend_m;
        nonfin |= o.nonfinite;
        // front: first x >= x0 - 1 (<= nx - 2) with a + to - crossing
        if (x >= max(x0 - 1, 0) && x <= nx - 2) {
            const ColObs &o1 = c[x + 1];
            if (o.fl0 && o1.fl0 && o.phi0 > 0.f && o1.phi0 <= 0.f) atomicMin(&s_first[0], x);
            if (o.fl1 && o1.fl1 && o.phi1 > 0.f && o1.phi1 <= 0.f) atomicMin(&s_first[1], x);
        }
    }
    double area = 0, perim = 0, hsum = 0, de = 0, wl = 0, wu = 0;
    int closed = 0;
    const double yc = (ny - 1) / 2.0;
    for (int k = tid; k < ncap; k += blockDim.x) {
        const ColObs &o = c[x0 + k];
        const int b0 = w0[2 * k], t0 = w0[2 * k + 1];
        atomicMin(&s_min_h, o.h);
        hsum += o.h;
        double g;
        if (o.h == 0) {
            closed = 1;
            g = (ny - b0 - t0) / 2.0;
        } else {
            g = (double)max(o.b - b0, o.t - t0);
            wl += o.wet_lo;
            wu += o.wet_hi;
        }
        de = fmax(de, g);
        area += fmax(0.0, yc - (o.b - 0.5));
        perim += 1.0;
        if (k + 1 < ncap) perim += fabs((double)(c[x0 + k + 1].b - o.b));
    }
    ma = block_sum(ma, sh); mb = block_sum(mb, sh); mc = block_sum(mc, sh);
    mm = block_sum(mm, sh); pa = block_sum(pa, sh); pb = block_sum(pb, sh);
    pc = block_sum(pc, sh); pm = block_sum(pm, sh);
    area = block_sum(area, sh); perim = block_sum(perim, sh);
    hsum = block_sum(hsum, sh); wl = block_sum(wl, sh); wu = block_sum(wu, sh);
    // max of de, or of flags, by negated / summed reductions
    sh[tid] = de;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = fmax(sh[tid], sh[tid + s]);
        __syncthreads();
    }
    de = sh[0];
    __syncthreads();
    const double nclosed = block_sum((double)closed, sh);
    const double nnonfin = block_sum((double)nonfin, sh);
    if (tid == 0) {
        LbmObsDev r;
        r.step = t;
        int nnonfin_any = 0;
        double z[2];
        const int rows[2] = {(ny - 1) / 2, ny / 2};
        for (int k = 0; k < 2; ++k) {
            const int xf = s_first[k];
            if (xf == 0x7fffffff) {
                z[k] = nan("");
            } else {
                const float p0 = rows[k] == rows[0] ? c[xf].phi0 : c[xf].phi1;
                const float p1 = rows[k] == rows[0] ? c[xf + 1].phi0 : c[xf + 1].phi1;
                z[k] = xf + (double)p0 / ((double)p0 - (double)p1) - (x0 - 0.5);
            }
        }
        r.front = rows[0] == rows[1] ? z[0] : 0.5 * (z[0] + z[1]);
        r.wetted_lower = wl;
        r.wetted_upper = wu;
        r.r_min = ncap > 0 ? s_min_h / 2.0 : 0.0;
        r.r_ave = ncap > 0 ? hsum / ncap / 2.0 : 0.0;
        r.r_h = perim > 0 ? area / perim : 0.0;
        r.delta_e = de;
        const LatState s = st[l];
        if (sums) {
            // the updated nodes' content (the column pass left it out of
            // ma .. mc, which hold minus the nodes that turned solid)
            const double *q = sums + 3 * l;
            ma += q[0];
            mb += q[1];
            mc += q[2];
            if (!(q[0] + q[1] < 3.0e38)) nnonfin_any = 1;
        }
        r.ledger_a = s.ledger[0] + pa;
        r.ledger_b = s.ledger[1] + pb;
        r.ledger_c = s.ledger[2] + pc;
        r.ledger_m = s.ledger[3] + pm;
        r.precip_mass = mm + r.ledger_m;
        r.mass_a = ma;
        r.mass_b = mb;
        r.mass_c = mc;
        r.closed = nclosed > 0;
        r.nonfinite = (nnonfin > 0) || nnonfin_any || s.nonfinite;
        r.closure_step = s.closure == ~0ull ? -1 : (long long)s.closure;
        out[l] = r;
    }
}

}  // namespace lbmk
