// lbm_static.cu -- lbm_observables_static: the observables of one lattice
// held in caller-owned device buffers, computed without allocating memory.
//
// Some callers cannot allocate device memory: code running inside a memory
// pool or arena that another runtime owns (a framework's caching
// allocator, an embedded or safety-certified build that forbids dynamic
// allocation after start-up), or code that must not synchronize the
// device, which cudaMalloc and cudaFree may do.  They cannot create a
// handle either, since lbm_create allocates.  This entry point takes the
// lattice state as device pointers and writes the result to a device
// pointer; its only working memory is the file-scope array below, of a
// fixed maximum size, that every GPU loading this library holds until the
// process exits.
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbmk {

// Per-column partial results of one call (a column's fluid content, wall
// profile and centerline values).  Every call writes all entries it later
// reads, so nothing has to be cleared between calls.
struct StaticCol {
    double mass_a, mass_b, mass_c, mass_m;
    float phi0, phi1;
    int32_t h, b, t, b0, t0;
    int32_t wet_lo, wet_hi, fl0, fl1, nonfinite;
};

constexpr int kStaticMaxColumns = LBM_STATIC_MAX_COLUMNS;

// The scratch shared by every call on a device.  In host code this name is
// only a stand-in: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) StaticCol g_static_cols[kStaticMaxColumns];

// One thread per column: walks the column of the canonical state
// (post-streaming populations [22][ny][nx], current and initial masks,
// deposit) and records its partial results.
__global__ void k_static_columns(const float *__restrict__ pops,
                                 const uint8_t *__restrict__ solid,
                                 const uint8_t *__restrict__ solid0,
                                 const double *__restrict__ dep, int nx,
                                 int ny, StaticCol *__restrict__ cols) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const int64_t P = (int64_t)nx * ny;
    const int yc0 = (ny - 1) / 2, yc1 = ny / 2;
    StaticCol o = {};
    int lo = -1, b = 0, t = 0, b0 = 0, t0 = 0;
    bool below = true, below0 = true;
    for (int y = 0; y < ny; ++y) {
        const int64_t n = (int64_t)y * nx + x;
        if (solid0[n]) {
            if (below0) ++b0;
            ++t0;
        } else {
            below0 = false;
            t0 = 0;
        }
        if (solid[n]) {
            if (below) ++b;
            ++t;
            continue;
        }
        below = false;
        t = 0;
        float ra = 0.f, rb = 0.f;
        for (int i = 0; i < Q; ++i) {
            ra += pops[i * P + n];
            rb += pops[(Q + i) * P + n];
        }
        const float c = pops[18 * P + n] + pops[19 * P + n] + pops[20 * P + n] +
                        pops[21 * P + n];
        if (!(ra + rb < 3.0e38f)) o.nonfinite = 1;
        o.mass_a += ra;
        o.mass_b += rb;
        o.mass_c += c;
        o.mass_m += dep[n];
        o.h += 1;
        if (lo < 0) { lo = y; o.wet_lo = ra > rb; }
        o.wet_hi = ra > rb;
        if (y == yc0) { o.phi0 = ra - rb; o.fl0 = 1; }
        if (y == yc1) { o.phi1 = ra - rb; o.fl1 = 1; }
    }
    o.b = o.h == 0 ? ny : b;
    o.t = o.h == 0 ? ny : t;
    if (o.h == 0) o.wet_lo = o.wet_hi = 0;
    o.b0 = b0;
    o.t0 = t0;
    cols[x] = o;
}

__device__ __forceinline__ double static_block_sum(double v, double *sh) {
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

struct StaticBook {
    double ledger[4];
    long long step, closure_step;
    int nx, ny, cap_x0, cap_x1;
};

// One block of 256 threads reduces the columns into *out.
__global__ void k_static_reduce(const StaticCol *__restrict__ c,
                                StaticBook bk, lbm_obs *out) {
    __shared__ double sh[256];
    __shared__ int s_first[2];
    __shared__ int s_min_h;
    const int tid = threadIdx.x;
    const int nx = bk.nx, ny = bk.ny, x0 = bk.cap_x0, x1 = bk.cap_x1;
    const int ncap = x1 - x0;
    if (tid == 0) { s_first[0] = s_first[1] = 0x7fffffff; s_min_h = 0x7fffffff; }
    __syncthreads();
    double ma = 0, mb = 0, mc = 0, mm = 0;
    int nonfin = 0;
    for (int x = tid; x < nx; x += blockDim.x) {
        const StaticCol &o = c[x];
        ma += o.mass_a; mb += o.mass_b; mc += o.mass_c; mm += o.mass_m;
        nonfin |= o.nonfinite;
        if (x >= max(x0 - 1, 0) && x <= nx - 2) {
            const StaticCol &o1 = c[x + 1];
            if (o.fl0 && o1.fl0 && o.phi0 > 0.f && o1.phi0 <= 0.f) atomicMin(&s_first[0], x);
            if (o.fl1 && o1.fl1 && o.phi1 > 0.f && o1.phi1 <= 0.f) atomicMin(&s_first[1], x);
        }
    }
    double area = 0, perim = 0, hsum = 0, de = 0, wl = 0, wu = 0;
    int closed = 0;
    const double yc = (ny - 1) / 2.0;
    for (int k = tid; k < ncap; k += blockDim.x) {
        const StaticCol &o = c[x0 + k];
        atomicMin(&s_min_h, o.h);
        hsum += o.h;
        double g;
        if (o.h == 0) {
            closed = 1;
            g = (ny - o.b0 - o.t0) / 2.0;
        } else {
            g = (double)max(o.b - o.b0, o.t - o.t0);
            wl += o.wet_lo;
            wu += o.wet_hi;
        }
        de = fmax(de, g);
        area += fmax(0.0, yc - (o.b - 0.5));
        perim += 1.0;
        if (k + 1 < ncap) perim += fabs((double)(c[x0 + k + 1].b - o.b));
    }
    ma = static_block_sum(ma, sh); mb = static_block_sum(mb, sh);
    mc = static_block_sum(mc, sh); mm = static_block_sum(mm, sh);
    area = static_block_sum(area, sh); perim = static_block_sum(perim, sh);
    hsum = static_block_sum(hsum, sh); wl = static_block_sum(wl, sh);
    wu = static_block_sum(wu, sh);
    sh[tid] = de;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) sh[tid] = fmax(sh[tid], sh[tid + s]);
        __syncthreads();
    }
    de = sh[0];
    __syncthreads();
    const double nclosed = static_block_sum((double)closed, sh);
    const double nnonfin = static_block_sum((double)nonfin, sh);
    if (tid == 0) {
        lbm_obs r;
        r.step = bk.step;
        double z[2];
        const int rows[2] = {(ny - 1) / 2, ny / 2};
        for (int k = 0; k < 2; ++k) {
            const int xf = s_first[k];
            if (xf == 0x7fffffff) {
                z[k] = nan("");
            } else {
                const float p0 = k == 0 ? c[xf].phi0 : c[xf].phi1;
                const float p1 = k == 0 ? c[xf + 1].phi0 : c[xf + 1].phi1;
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
        r.ledger_a = bk.ledger[0];
        r.ledger_b = bk.ledger[1];
        r.ledger_c = bk.ledger[2];
        r.ledger_m = bk.ledger[3];
        r.precip_mass = mm + bk.ledger[3];
        r.mass_a = ma;
        r.mass_b = mb;
        r.mass_c = mc;
        r.closed = nclosed > 0;
        r.nonfinite = nnonfin > 0;
        r.closure_step = bk.closure_step;
        *out = r;
    }
}

}  // namespace lbmk

using namespace lbmk;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
StaticCol *g_static_ptr[kMaxDevices] = {};
}  // namespace

extern "C" lbm_status lbm_observables_static(
    const float *pops, const uint8_t *solid, const uint8_t *solid0,
    const double *deposit, int32_t nx, int32_t ny, int32_t cap_x0,
    int32_t cap_x1, const double ledger[4], int64_t step,
    int64_t closure_step, lbm_obs *out, void *cuda_stream) {
    if (!pops || !solid || !solid0 || !deposit || !ledger || !out)
        return LBM_EINVAL;
    if (nx < 1 || ny < 3 || nx > kStaticMaxColumns)
        return LBM_EINVAL;
    if (!(0 <= cap_x0 && cap_x0 < cap_x1 && cap_x1 <= nx)) return LBM_EINVAL;
    if ((int64_t)NPOP * nx * ny >= ((int64_t)1 << 31)) return LBM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return LBM_ECUDA;
    StaticCol *cols = nullptr;
    {
        // First call on this device (made current by the caller): look up
        // the device address of the scratch array.
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_cols) != cudaSuccess || !p)
                return LBM_ECUDA;
            g_static_ptr[dev] = static_cast<StaticCol *>(p);
        }
        cols = g_static_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    StaticBook bk;
    for (int k = 0; k < 4; ++k) bk.ledger[k] = ledger[k];
    bk.step = step;
    bk.closure_step = closure_step;
    bk.nx = nx;
    bk.ny = ny;
    bk.cap_x0 = cap_x0;
    bk.cap_x1 = cap_x1;
    // an error left pending by earlier, unrelated work is not this call's:
    // report it without launching (and without clearing it)
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
    k_static_columns<<<(nx + 127) / 128, 128, 0, s>>>(pops, solid, solid0,
                                                      deposit, nx, ny, cols);
    k_static_reduce<<<1, 256, 0, s>>>(cols, bk, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
