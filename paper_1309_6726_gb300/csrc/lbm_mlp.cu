// lbm_mlp.cu -- the surrogate network of lbm_mlp.h: forward, backward and
// Adam kernels.  Every matrix product is one launch of gemm_bf16: BF16
// operands staged in shared memory, tensor-core mma.sync (m16n8k16, FP32
// accumulate), and a fused epilogue (bias, tanh, or the tanh derivative of
// back-propagation).  Operands are read through (row, column) strides, so
// the transposed products of the backward pass need no transposed copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm_mlp.h"

namespace lbmmlp {

constexpr int BM = 64, BN = 64, BK = 32, KP = BK + 8;  // KP: padded row
constexpr int GEMM_THREADS = 128;                        // 2 x 2 warps
constexpr int kSplit = 8;  // K split of the weight-gradient products

enum Epi : int {
    EPI_PLAIN = 0,      // C = A B
    EPI_BIAS = 1,       // C = A B + bias[n]
    EPI_BIAS_TANH = 2,  // C = tanh(A B + bias[n])
    EPI_DTANH = 3,      // C = (A B) (1 - H[m][n]^2)
};

template <class T>
__device__ __forceinline__ __nv_bfloat16 to_bf16(T v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_bf16<float>(float v) {
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_bf16<__nv_bfloat16>(__nv_bfloat16 v) {
    return v;
}

__device__ __forceinline__ void mma_bf16(float d[4], const unsigned a[4],
                                         const unsigned b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] (row stride ldc) = epilogue(sum_k A(m, k) B(k, n)), m < M, n < N,
// with A(m, k) = a[m * sam + k * sak] and B(k, n) = b[k * sbk + n * sbn],
// both rounded to BF16 on their way into shared memory.  Split K
// (EPI_PLAIN only): block z sums k in [z kchunk, (z + 1) kchunk) and writes
// its partial product to c + z * M * ldc (k_sum_parts adds them up).
template <class TA, class TB>
__global__ void __launch_bounds__(GEMM_THREADS)
    gemm_bf16(int M, int N, int K, const TA *__restrict__ a, long sam,
              long sak, const TB *__restrict__ b, long sbk, long sbn,
              float *__restrict__ c, long ldc, int epi,
              const float *__restrict__ bias, const float *__restrict__ h,
              long ldh, int kchunk) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][KP];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][KP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t4 = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    float acc[2][4][4] = {};
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    c += (long)blockIdx.z * M * ldc;
    for (int k0 = kb; k0 < ke; k0 += BK) {
        // A tile, BM x BK: walk the unit-stride index fastest
        if (sak == 1) {
#pragma unroll 2
            for (int j = 0; j < BM * BK / GEMM_THREADS; ++j) {
                const int e = tid + j * GEMM_THREADS;
                const int kk = e % BK, mm = e / BK;
                const int m = m0 + mm, k = k0 + kk;
                As[mm][kk] = (m < M && k < ke) ? to_bf16(a[m * sam + k]) : zero;
            }
        } else {
#pragma unroll 2
            for (int j = 0; j < BM * BK / GEMM_THREADS; ++j) {
                const int e = tid + j * GEMM_THREADS;
                const int mm = e % BM, kk = e / BM;
                const int m = m0 + mm, k = k0 + kk;
                As[mm][kk] = (m < M && k < ke) ? to_bf16(a[m * sam + k * sak]) : zero;
            }
        }
        // B tile, BK x BN, kept n-major: Bs[n][k]
        if (sbn == 1) {
#pragma unroll 2
            for (int j = 0; j < BN * BK / GEMM_THREADS; ++j) {
                const int e = tid + j * GEMM_THREADS;
                const int nn = e % BN, kk = e / BN;
                const int n = n0 + nn, k = k0 + kk;
                Bs[nn][kk] = (n < N && k < ke) ? to_bf16(b[k * sbk + n]) : zero;
            }
        } else {
#pragma unroll 2
            for (int j = 0; j < BN * BK / GEMM_THREADS; ++j) {
                const int e = tid + j * GEMM_THREADS;
                const int kk = e % BK, nn = e / BK;
                const int n = n0 + nn, k = k0 + kk;
                Bs[nn][kk] = (n < N && k < ke) ? to_bf16(b[k * sbk + n * sbn]) : zero;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm * 32 + mi * 16 + g;
                af[mi][0] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * t4]);
                af[mi][1] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * t4]);
                af[mi][2] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * t4 + 8]);
                af[mi][3] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int cidx = wn * 32 + ni * 8 + g;
                bfr[ni][0] = *reinterpret_cast<const unsigned *>(&Bs[cidx][kk + 2 * t4]);
                bfr[ni][1] = *reinterpret_cast<const unsigned *>(&Bs[cidx][kk + 2 * t4 + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm * 32 + mi * 16 + g + (q >> 1) * 8;
                const int n = n0 + wn * 32 + ni * 8 + 2 * t4 + (q & 1);
                if (m >= M || n >= N) continue;
                float v = acc[mi][ni][q];
                if (epi == EPI_BIAS || epi == EPI_BIAS_TANH) v += bias[n];
                if (epi == EPI_BIAS_TANH) v = tanhf(v);
                if (epi == EPI_DTANH) {
                    const float hv = h[m * ldh + n];
                    v *= 1.0f - hv * hv;
                }
                c[m * ldc + n] = v;
            }
}

// c[i] = sum over z of parts[z * n + i], in order z = 0, 1, ...
__global__ void k_sum_parts(const float *__restrict__ parts, int nparts,
                            long n, float *__restrict__ c) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < nparts; ++z) v += parts[z * n + i];
        c[i] = v;
    }
}

// dy = 2 (y - t) / (rows * cols) where t is a number, 0 where t is NaN;
// *loss += sum of (y - t)^2 / (rows * cols) over the numbers.
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t,
                      long n, float inv_count, float *__restrict__ dy,
                      double *__restrict__ loss) {
    __shared__ double sh[256];
    double s = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        const float tv = t[i];
        float d = 0.f;
        if (!isnan(tv)) {
            d = y[i] - tv;
            s += (double)d * d;
        }
        dy[i] = 2.0f * d * inv_count;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0] * inv_count);
}

// db[n] = sum_m dz[m][n] for an M x N row-major matrix.
__global__ void k_colsum(const float *__restrict__ dz, int M, int N,
                         float *__restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += dz[(long)m * N + n];
    db[n] = s;
}

// Adam with bias correction; refreshes the BF16 copy.
__global__ void k_adam(float *__restrict__ w, __nv_bfloat16 *__restrict__ wb,
                       const float *__restrict__ gr, float *__restrict__ m1,
                       float *__restrict__ m2, long n, float lr, float c1,
                       float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        const float gv = gr[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gv;
        const float v = b2 * m2[i] + (1.0f - b2) * gv * gv;
        m1[i] = a;
        m2[i] = v;
        const float wv = w[i] - lr * (a * c1) / (sqrtf(v * c2) + eps);
        w[i] = wv;
        wb[i] = __float2bfloat16_rn(wv);
    }
}

__global__ void k_to_bf16(const float *__restrict__ w,
                          __nv_bfloat16 *__restrict__ wb, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(w[i]);
}

}  // namespace lbmmlp

using namespace lbmmlp;

struct lbm_mlp {
    lbm_mlp_shape sh{};
    long np = 0;
    std::vector<long> off_w, off_b;  // per layer (L + 1)
    float *w = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *wb = nullptr;
    std::vector<float *> hs;         // hidden activations, [max_batch][H]
    float *y = nullptr, *dy = nullptr, *dz[2] = {nullptr, nullptr};
    float *split = nullptr;  // split-K partial products of a weight gradient
    double *d_loss = nullptr;
    cudaStream_t own = nullptr, stream = nullptr;
    long adam_t = 0;
    std::string err;
    bool dead = false;
};

namespace {
std::string g_create_err;

lbm_status fail(lbm_mlp *h, lbm_status st, const std::string &msg) {
    if (h) {
        h->err = msg;
        if (st == LBM_ECUDA) h->dead = true;
    } else {
        g_create_err = msg;
    }
    return st;
}

#define MCK(h, call)                                                         \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess)                                               \
            return fail(h, LBM_ECUDA, std::string(#call) + ": " +            \
                                          cudaGetErrorString(e_));           \
    } while (0)

template <class TA, class TB>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const TA *a, long sam,
                 long sak, const TB *b, long sbk, long sbn, float *c, long ldc,
                 int epi, const float *bias = nullptr,
                 const float *hh = nullptr, long ldh = 0) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    gemm_bf16<TA, TB><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, a, sam, sak, b,
                                                    sbk, sbn, c, ldc, epi,
                                                    bias, hh, ldh, K);
    return cudaGetLastError();
}

// C = A B (M x N, row stride N) with K split over `parts` blocks of
// columns-of-work when the plain grid is small; the partial products go to
// `scratch` (parts * M * N floats) and are added in a fixed order.
template <class TA, class TB>
cudaError_t gemm_split(cudaStream_t s, int M, int N, int K, const TA *a,
                       long sam, long sak, const TB *b, long sbk, long sbn,
                       float *c, float *scratch, int parts) {
    const int kchunk = ((K + parts - 1) / parts + BK - 1) / BK * BK;
    parts = (K + kchunk - 1) / kchunk;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, parts);
    gemm_bf16<TA, TB><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, a, sam, sak, b,
                                                    sbk, sbn, scratch, (long)N,
                                                    EPI_PLAIN, nullptr, nullptr,
                                                    0, kchunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long n = (long)M * N;
    k_sum_parts<<<(int)std::min<long>((n + 255) / 256, 1024), 256, 0, s>>>(
        scratch, parts, n, c);
    return cudaGetLastError();
}

int n_layers_total(const lbm_mlp *h) { return h->sh.n_layers + 1; }
int in_of(const lbm_mlp *h, int l) { return l == 0 ? h->sh.n_in : h->sh.n_hidden; }
int out_of(const lbm_mlp *h, int l) {
    return l == h->sh.n_layers ? h->sh.n_out : h->sh.n_hidden;
}

// Forward pass into the handle's activations; the output lands in y_out.
cudaError_t forward(lbm_mlp *h, const float *x, int batch, float *y_out) {
    const int L = h->sh.n_layers;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l <= L && e == cudaSuccess; ++l) {
        const int K = in_of(h, l), N = out_of(h, l);
        const float *in = l == 0 ? x : h->hs[l - 1];
        float *out = l == L ? y_out : h->hs[l];
        e = gemm(h->stream, batch, N, K, in, (long)K, 1L, h->wb + h->off_w[l],
                 1L, (long)K, out, (long)N, l == L ? EPI_BIAS : EPI_BIAS_TANH,
                 h->w + h->off_b[l]);
    }
    return e;
}

// Backward pass from dy (in h->dy) into h->grad.
cudaError_t backward(lbm_mlp *h, const float *x, int batch) {
    const int L = h->sh.n_layers, H = h->sh.n_hidden;
    const float *dzl = h->dy;  // gradient at the pre-activation of layer l
    int cur = 0;
    cudaError_t e = cudaSuccess;
    for (int l = L; l >= 0 && e == cudaSuccess; --l) {
        const int K = in_of(h, l), N = out_of(h, l);
        const float *in = l == 0 ? x : h->hs[l - 1];
        // dW_l[n][k] = sum_b dz[b][n] in[b][k]: a small output and a long
        // sum over the batch, split into kSplit parts
        e = gemm_split(h->stream, N, K, batch, dzl, 1L, (long)N, in, (long)K,
                       1L, h->grad + h->off_w[l], h->split, kSplit);
        if (e != cudaSuccess) break;
        k_colsum<<<(N + 127) / 128, 128, 0, h->stream>>>(dzl, batch, N,
                                                         h->grad + h->off_b[l]);
        e = cudaGetLastError();
        if (e != cudaSuccess || l == 0) break;
        // dz_{l-1}[b][k] = (sum_n dz[b][n] W_l[n][k]) (1 - h_{l-1}[b][k]^2)
        float *next = h->dz[cur];
        e = gemm(h->stream, batch, K, N, dzl, (long)N, 1L, h->wb + h->off_w[l],
                 (long)K, 1L, next, (long)K, EPI_DTANH, nullptr, h->hs[l - 1],
                 (long)H);
        dzl = next;
        cur ^= 1;
    }
    return e;
}

lbm_status check_batch(lbm_mlp *h, int batch) {
    if (!h) return LBM_EINVAL;
    if (h->dead) return LBM_ECUDA;
    if (batch < 1 || batch > h->sh.max_batch)
        return fail(h, LBM_EINVAL, "batch outside 1..max_batch");
    return LBM_OK;
}

// loss and dy from the forward output in h->y
lbm_status loss_and_dy(lbm_mlp *h, const float *target, int batch) {
    const long n = (long)batch * h->sh.n_out;
    MCK(h, cudaMemsetAsync(h->d_loss, 0, sizeof(double), h->stream));
    k_mse<<<(int)std::min<long>((n + 255) / 256, 1024), 256, 0, h->stream>>>(
        h->y, target, n, 1.0f / (float)n, h->dy, h->d_loss);
    MCK(h, cudaGetLastError());
    return LBM_OK;
}

lbm_status read_loss(lbm_mlp *h, double *loss) {
    if (!loss) return LBM_OK;
    MCK(h, cudaMemcpyAsync(loss, h->d_loss, sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
    MCK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_mlp_create(const lbm_mlp_shape *shape, lbm_mlp **out) {
    if (!shape || !out) return fail(nullptr, LBM_EINVAL, "NULL argument");
    *out = nullptr;
    const lbm_mlp_shape s = *shape;
    if (s.n_in < 1 || s.n_in > 256 || s.n_hidden < 16 || s.n_hidden > 1024 ||
        s.n_hidden % 16 != 0 || s.n_layers < 1 || s.n_layers > 8 ||
        s.n_out < 1 || s.n_out > 1024 || s.max_batch < 1 ||
        s.max_batch > (1 << 24))
        return fail(nullptr, LBM_EINVAL, "shape outside the supported ranges");
    lbm_mlp *h = new (std::nothrow) lbm_mlp();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation");
    h->sh = s;
    long np = 0;
    for (int l = 0; l <= s.n_layers; ++l) {
        h->off_w.push_back(np);
        np += (long)out_of(h, l) * in_of(h, l);
        h->off_b.push_back(np);
        np += out_of(h, l);
    }
    h->np = np;
    bool ok = true;
    auto al = [&](auto **p, size_t n) {
        if (ok && cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(**p)) != cudaSuccess) ok = false;
    };
    al(&h->w, np);
    al(&h->grad, np);
    al(&h->m1, np);
    al(&h->m2, np);
    al(&h->wb, np);
    h->hs.assign(s.n_layers, nullptr);
    for (auto &p : h->hs) al(&p, (size_t)s.max_batch * s.n_hidden);
    al(&h->y, (size_t)s.max_batch * s.n_out);
    al(&h->dy, (size_t)s.max_batch * s.n_out);
    al(&h->dz[0], (size_t)s.max_batch * s.n_hidden);
    al(&h->dz[1], (size_t)s.max_batch * s.n_hidden);
    al(&h->d_loss, 1);
    {
        long wmax = 0;  // largest weight matrix
        for (int l = 0; l <= s.n_layers; ++l)
            wmax = std::max(wmax, (long)out_of(h, l) * in_of(h, l));
        al(&h->split, (size_t)kSplit * wmax);
    }
    if (ok && cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess)
        ok = false;
    h->stream = h->own;
    if (ok) {
        for (void *p : {(void *)h->w, (void *)h->grad, (void *)h->m1, (void *)h->m2})
            ok = ok && cudaMemset(p, 0, np * sizeof(float)) == cudaSuccess;
        ok = ok && cudaMemset(h->wb, 0, np * sizeof(__nv_bfloat16)) == cudaSuccess;
    }
    if (!ok) {
        lbm_mlp_destroy(h);
        return fail(nullptr, LBM_ENOMEM, "device allocation");
    }
    *out = h;
    return LBM_OK;
}

int64_t lbm_mlp_param_count(const lbm_mlp *h) { return h ? h->np : -1; }

lbm_status lbm_mlp_set_params(lbm_mlp *h, const float *host, int64_t n) {
    if (!h || !host) return LBM_EINVAL;
    if (h->dead) return LBM_ECUDA;
    if (n != h->np) return fail(h, LBM_EINVAL, "parameter count mismatch");
    MCK(h, cudaMemcpyAsync(h->w, host, n * sizeof(float), cudaMemcpyHostToDevice,
                           h->stream));
    MCK(h, cudaMemsetAsync(h->m1, 0, n * sizeof(float), h->stream));
    MCK(h, cudaMemsetAsync(h->m2, 0, n * sizeof(float), h->stream));
    k_to_bf16<<<(int)std::min<long>((n + 255) / 256, 4096), 256, 0, h->stream>>>(
        h->w, h->wb, n);
    MCK(h, cudaGetLastError());
    // the host array may be reused as soon as this returns
    MCK(h, cudaStreamSynchronize(h->stream));
    h->adam_t = 0;
    return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp *h, float *host, int64_t n) {
    if (!h || !host) return LBM_EINVAL;
    if (h->dead) return LBM_ECUDA;
    if (n != h->np) return fail(h, LBM_EINVAL, "parameter count mismatch");
    MCK(h, cudaMemcpyAsync(host, h->w, n * sizeof(float), cudaMemcpyDeviceToHost,
                           h->stream));
    MCK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_set_stream(lbm_mlp *h, void *cuda_stream) {
    if (!h) return LBM_EINVAL;
    h->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->own;
    return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp *h, const float *x, int32_t batch, float *y) {
    lbm_status st = check_batch(h, batch);
    if (st != LBM_OK) return st;
    if (!x || !y) return fail(h, LBM_EINVAL, "NULL argument");
    MCK(h, forward(h, x, batch, y));
    return LBM_OK;
}

lbm_status lbm_mlp_grad(lbm_mlp *h, const float *x, const float *target,
                        int32_t batch, float *grad, double *loss) {
    lbm_status st = check_batch(h, batch);
    if (st != LBM_OK) return st;
    if (!x || !target || !grad) return fail(h, LBM_EINVAL, "NULL argument");
    MCK(h, forward(h, x, batch, h->y));
    if ((st = loss_and_dy(h, target, batch)) != LBM_OK) return st;
    MCK(h, backward(h, x, batch));
    MCK(h, cudaMemcpyAsync(grad, h->grad, h->np * sizeof(float),
                           cudaMemcpyDeviceToDevice, h->stream));
    return read_loss(h, loss);
}

lbm_status lbm_mlp_train_step(lbm_mlp *h, const float *x, const float *target,
                              int32_t batch, float lr, double *loss) {
    lbm_status st = check_batch(h, batch);
    if (st != LBM_OK) return st;
    if (!x || !target) return fail(h, LBM_EINVAL, "NULL argument");
    if (!(lr > 0.f)) return fail(h, LBM_EINVAL, "learning rate must be > 0");
    MCK(h, forward(h, x, batch, h->y));
    if ((st = loss_and_dy(h, target, batch)) != LBM_OK) return st;
    MCK(h, backward(h, x, batch));
    ++h->adam_t;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)h->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)h->adam_t)));
    k_adam<<<(int)std::min<long>((h->np + 255) / 256, 4096), 256, 0, h->stream>>>(
        h->w, h->wb, h->grad, h->m1, h->m2, h->np, lr, c1, c2);
    MCK(h, cudaGetLastError());
    return read_loss(h, loss);
}

void lbm_mlp_destroy(lbm_mlp *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *p : {(void *)h->w, (void *)h->grad, (void *)h->m1, (void *)h->m2,
                    (void *)h->wb, (void *)h->y, (void *)h->dy,
                    (void *)h->dz[0], (void *)h->dz[1], (void *)h->d_loss,
                    (void *)h->split})
        if (p) cudaFree(p);
    for (float *p : h->hs)
        if (p) cudaFree(p);
    if (h->own) cudaStreamDestroy(h->own);
    delete h;
}

const char *lbm_mlp_last_error(const lbm_mlp *h) {
    return h ? h->err.c_str() : g_create_err.c_str();
}

}  // extern "C"
