// qt_router.cu -- the learned router of the router form (a start cell for the
// nearest-cell searches of Algorithm III, Pages & Wilbertz, arXiv:1101.3228,
// Sec. 3.2; the paper's kd-tree attempt there is the prior art for a
// sub-linear search): its tables and its training.  The search itself is in
// qt_router_search.cu.
//
// Router: MLP d -> 64 -> 64 -> 64 (ReLU) on whitened coordinates
// z = L_k^{-1}(x - mu_k); the output is one of 64 buckets, a k-means partition
// of the grid points (the same index partition for every layer, since the
// grids of the layers are images of one base grid).
// Training: pairs drawn by the library's sampler, labelled with the bucket of
// their exact cell (the library's own certified search), cross-entropy with
// Adam, forward and backward passes in FP32 on the CUDA cores.
// Elkan tables: per grid point its C nearest other points in increasing
// distance (FP64 distances rounded down), the lists the certified walk scans.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/qt.h"
#include "qt_forward.cuh"
#include "qt_launch.h"

using namespace qt;

struct qt_router {
    int device = 0;
    int d = 0, n = 0, N = 0, C = 0;
    long long P = 0;
    float* params = nullptr;       // dev, packed
    float* linv = nullptr;         // dev [n+1][d][d]
    int32_t* bstart = nullptr;     // dev [65]
    int32_t* members = nullptr;    // dev [N]
    int32_t* nb_idx = nullptr;     // dev [n+1][N][C]
    float* nb_dist = nullptr;      // dev [n+1][N][C]
    unsigned long long checksum = 0;
    qt_router_info info{};
};

namespace qt {

// ------------------------------------------------------------------ checksum of the grids

__global__ void grid_checksum_kernel(const double* __restrict__ g, long long count, unsigned long long* out)
{
    unsigned long long acc = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(g[e]);
        acc += b * (2ull * (unsigned long long)e + 1ull);   // position-weighted, order independent
    }
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// ------------------------------------------------------------------ MLP training (FP32, CUDA cores)

// Training forward + loss: writes h1, h2 and dlogits = (softmax - onehot) / B.
template <int DM>
__global__ void __launch_bounds__(128) mlp_train_forward_kernel(const float* __restrict__ P, int d,
                                                                const float* __restrict__ Z,
                                                                const int32_t* __restrict__ lab, int B,
                                                                float* H1, float* H2, float* DL, double* loss,
                                                                int* correct)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float* W1 = P;
    const float* b1 = W1 + kRtHidden * d;
    const float* W2 = b1 + kRtHidden;
    const float* b2 = W2 + kRtHidden * kRtHidden;
    const float* W3 = b2 + kRtHidden;
    const float* b3 = W3 + kRtHidden * kRtHidden;
    float z[DM];
#pragma unroll
    for (int l = 0; l < DM; ++l) z[l] = l < d ? Z[(long long)b * d + l] : 0.0f;
    float h[kRtHidden], g[kRtHidden];
#pragma unroll
    for (int o = 0; o < kRtHidden; ++o) {
        float a = b1[o];
#pragma unroll
        for (int l = 0; l < DM; ++l)
            if (l < d) a = fmaf(W1[o * d + l], z[l], a);
        h[o] = fmaxf(a, 0.0f);
        H1[(long long)b * kRtHidden + o] = h[o];
    }
#pragma unroll
    for (int o = 0; o < kRtHidden; ++o) g[o] = b2[o];
    for (int i = 0; i < kRtHidden; ++i) {
        const float hi = h[i];
#pragma unroll
        for (int o = 0; o < kRtHidden; ++o) g[o] = fmaf(W2[o * kRtHidden + i], hi, g[o]);
    }
#pragma unroll
    for (int o = 0; o < kRtHidden; ++o) {
        g[o] = fmaxf(g[o], 0.0f);
        H2[(long long)b * kRtHidden + o] = g[o];
    }
#pragma unroll
    for (int o = 0; o < kRtBuckets; ++o) h[o] = b3[o];     // h now holds the logits
    for (int i = 0; i < kRtHidden; ++i) {
        const float gi = g[i];
#pragma unroll
        for (int o = 0; o < kRtBuckets; ++o) h[o] = fmaf(W3[o * kRtHidden + i], gi, h[o]);
    }
    float mx = h[0];
    int am = 0;
#pragma unroll
    for (int o = 1; o < kRtBuckets; ++o)
        if (h[o] > mx) {
            mx = h[o];
            am = o;
        }
    float sum = 0.0f;
#pragma unroll
    for (int o = 0; o < kRtBuckets; ++o) sum += expf(h[o] - mx);
    const int y = lab[b];
    loss[b] = (double)(logf(sum) + mx - h[y]);
    correct[b] = am == y;
    const float inv = 1.0f / (sum * (float)B);
#pragma unroll
    for (int o = 0; o < kRtBuckets; ++o)
        DL[(long long)b * kRtBuckets + o] = expf(h[o] - mx) * inv - (o == y ? 1.0f / (float)B : 0.0f);
}

// Back-propagation to the hidden layers: dH2 = (W3^T dL) * [h2 > 0], dH1 = (W2^T dH2) * [h1 > 0].
__global__ void __launch_bounds__(128) mlp_train_backward_kernel(const float* __restrict__ P, int d, int B,
                                                                 const float* __restrict__ H1,
                                                                 const float* __restrict__ H2,
                                                                 const float* __restrict__ DL, float* DH1,
                                                                 float* DH2)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float* W2 = P + kRtHidden * d + kRtHidden;
    const float* W3 = W2 + kRtHidden * kRtHidden + kRtHidden;
    float g2[kRtHidden];
    for (int i = 0; i < kRtHidden; ++i) {
        float a = 0.0f;
        for (int o = 0; o < kRtBuckets; ++o) a = fmaf(W3[o * kRtHidden + i], DL[(long long)b * kRtBuckets + o], a);
        g2[i] = H2[(long long)b * kRtHidden + i] > 0.0f ? a : 0.0f;
        DH2[(long long)b * kRtHidden + i] = g2[i];
    }
    for (int i = 0; i < kRtHidden; ++i) {
        float a = 0.0f;
        for (int o = 0; o < kRtHidden; ++o) a = fmaf(W2[o * kRtHidden + i], g2[o], a);
        DH1[(long long)b * kRtHidden + i] = H1[(long long)b * kRtHidden + i] > 0.0f ? a : 0.0f;
    }
}

// Parameter gradients, one thread per parameter, batch summed in order.
__global__ void mlp_param_grad_kernel(int d, int B, const float* __restrict__ Z, const float* __restrict__ H1,
                                      const float* __restrict__ H2, const float* __restrict__ DL,
                                      const float* __restrict__ DH1, const float* __restrict__ DH2, float* G)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nW1 = kRtHidden * d, nb = kRtHidden, nW = kRtHidden * kRtHidden;
    const int total = nW1 + nb + 2 * (nW + nb);
    if (t >= total) return;
    float acc = 0.0f;
    int r = t;
    if (r < nW1) {
        const int o = r / d, l = r % d;
        for (int b = 0; b < B; ++b) acc = fmaf(DH1[(long long)b * kRtHidden + o], Z[(long long)b * d + l], acc);
    } else if ((r -= nW1) < nb) {
        for (int b = 0; b < B; ++b) acc += DH1[(long long)b * kRtHidden + r];
    } else if ((r -= nb) < nW) {
        const int o = r / kRtHidden, i = r % kRtHidden;
        for (int b = 0; b < B; ++b)
            acc = fmaf(DH2[(long long)b * kRtHidden + o], H1[(long long)b * kRtHidden + i], acc);
    } else if ((r -= nW) < nb) {
        for (int b = 0; b < B; ++b) acc += DH2[(long long)b * kRtHidden + r];
    } else if ((r -= nb) < nW) {
        const int o = r / kRtHidden, i = r % kRtHidden;
        for (int b = 0; b < B; ++b)
            acc = fmaf(DL[(long long)b * kRtBuckets + o], H2[(long long)b * kRtHidden + i], acc);
    } else {
        r -= nW;
        for (int b = 0; b < B; ++b) acc += DL[(long long)b * kRtBuckets + r];
    }
    G[t] = acc;
}

__global__ void adam_kernel(int P, float* w, const float* g, float* m, float* v, float lr, float b1t, float b2t)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P) return;
    const float gt = g[t];
    m[t] = 0.9f * m[t] + 0.1f * gt;
    v[t] = 0.999f * v[t] + 0.001f * gt * gt;
    const float mh = m[t] / (1.0f - b1t), vh = v[t] / (1.0f - b2t);
    w[t] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// Training draws of layer k: X = m_k + L_k z from the library's sampler (own
// stream: layer index 0x8000 + k), widened to FP64 for the exact search, and
// the whitened FP32 input z = L_k^{-1} (X - mu_k).
template <int DM>
__global__ void router_draw_kernel(int d, unsigned long long seed, int k, long long S, const float* __restrict__ pf,
                                   const float* __restrict__ mu, const float* __restrict__ linv, double* X64,
                                   float* Z)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S) return;
    float X[DM], Y[DM];
    pair_f32<DM>(pf, d, seed, 0x8000 + k, (unsigned long long)t, X, Y);
    float c[DM];
#pragma unroll
    for (int l = 0; l < DM; ++l) c[l] = l < d ? X[l] - mu[l] : 0.0f;
    for (int l = 0; l < d; ++l) {
        X64[t * d + l] = (double)X[l];
        float a = 0.0f;
        for (int q = 0; q <= l; ++q) a = fmaf(linv[l * d + q], c[q], a);
        Z[t * d + l] = a;
    }
}

__global__ void gather_labels_kernel(const int32_t* cells, const int32_t* bucket_of, long long S, int32_t* lab)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < S) lab[t] = bucket_of[cells[t]];
}

// Elkan table of grid g, point i (one CTA): the C nearest other points in
// increasing distance, distances computed in FP64 and rounded down to FP32.
// 64-bit keys (distance bits, index) sorted bitonically in shared memory.
__global__ void elkan_table_kernel(const double* __restrict__ grids, int d, int N, int C, int npow2,
                                   long long goff0, int32_t* nb_idx, float* nb_dist)
{
    extern __shared__ unsigned long long keys[];
    const int i = blockIdx.x;
    const int g = blockIdx.y;                 // grid index - 1 (grids 1..n)
    const double* G = grids + (goff0 + (long long)g * N) * d;
    const double* ci = G + (long long)i * d;
    for (int j = threadIdx.x; j < npow2; j += blockDim.x) {
        unsigned long long key = ~0ull;
        if (j < N && j != i) {
            double acc = 0.0;
            for (int l = 0; l < d; ++l) {
                const double t = ci[l] - G[(long long)j * d + l];
                acc = fma(t, t, acc);
            }
            const float df = __double2float_rd(sqrt(acc) * (1.0 - 0x1p-50));
            key = ((unsigned long long)__float_as_uint(df) << 32) | (unsigned)j;
        }
        keys[j] = key;
    }
    __syncthreads();
    for (int size = 2; size <= npow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < npow2 / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = keys[lo], b = keys[hi];
                if ((a > b) == up) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    const long long base = ((long long)(g + 1) * N + i) * C;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const unsigned long long key = c < N - 1 ? keys[c] : ~0ull;
        nb_idx[base + c] = key == ~0ull ? i : (int32_t)(key & 0xFFFFFFFFu);
        nb_dist[base + c] = key == ~0ull ? __int_as_float(0x7F800000) : __uint_as_float((unsigned)(key >> 32));
    }
}

cudaError_t launch_grid_checksum(const double* grids, long long count, unsigned long long* out, cudaStream_t st)
{
    grid_checksum_kernel<<<256, 256, 0, st>>>(grids, count, out);
    return cudaGetLastError();
}

void router_fill_params(const qt_router* r, ForwardParams& fp)
{
    fp.rt_params = r->params;
    fp.rt_linv = r->linv;
    fp.rt_bstart = r->bstart;
    fp.rt_members = r->members;
    fp.rt_nb_idx = r->nb_idx;
    fp.rt_nb_dist = r->nb_dist;
    fp.rt_C = r->C;
    fp.rt_N = r->N;
    fp.rt_checksum = r->checksum;
}

bool router_matches(const qt_router* r, int d, int n, const int64_t* N)
{
    if (!r || r->d != d || r->n != n) return false;
    for (int k = 1; k <= n; ++k)
        if (N[k] != r->N) return false;
    return true;
}

}  // namespace qt

// ------------------------------------------------------------------ host: training and tables

namespace {

template <int DM>
cudaError_t launch_train_forward(const float* P, int d, const float* Z, const int32_t* lab, int B, float* H1,
                                 float* H2, float* DL, double* loss, int* correct, cudaStream_t st)
{
    qt::mlp_train_forward_kernel<DM><<<(B + 127) / 128, 128, 0, st>>>(P, d, Z, lab, B, H1, H2, DL, loss, correct);
    return cudaGetLastError();
}

cudaError_t train_forward(int dm, const float* P, int d, const float* Z, const int32_t* lab, int B, float* H1,
                          float* H2, float* DL, double* loss, int* correct, cudaStream_t st)
{
    switch (dm) {
    case 2: return launch_train_forward<2>(P, d, Z, lab, B, H1, H2, DL, loss, correct, st);
    case 4: return launch_train_forward<4>(P, d, Z, lab, B, H1, H2, DL, loss, correct, st);
    case 6: return launch_train_forward<6>(P, d, Z, lab, B, H1, H2, DL, loss, correct, st);
    case 8: return launch_train_forward<8>(P, d, Z, lab, B, H1, H2, DL, loss, correct, st);
    case 10: return launch_train_forward<10>(P, d, Z, lab, B, H1, H2, DL, loss, correct, st);
    case 12: return launch_train_forward<12>(P, d, Z, lab, B, H1, H2, DL, loss, correct, st);
    default: return launch_train_forward<16>(P, d, Z, lab, B, H1, H2, DL, loss, correct, st);
    }
}

cudaError_t draw(int dm, int d, unsigned long long seed, int k, long long S, const float* pf, const float* mu,
                 const float* linv, double* X64, float* Z, cudaStream_t st)
{
    const unsigned nb = (unsigned)((S + 255) / 256);
    switch (dm) {
    case 2: qt::router_draw_kernel<2><<<nb, 256, 0, st>>>(d, seed, k, S, pf, mu, linv, X64, Z); break;
    case 4: qt::router_draw_kernel<4><<<nb, 256, 0, st>>>(d, seed, k, S, pf, mu, linv, X64, Z); break;
    case 6: qt::router_draw_kernel<6><<<nb, 256, 0, st>>>(d, seed, k, S, pf, mu, linv, X64, Z); break;
    case 8: qt::router_draw_kernel<8><<<nb, 256, 0, st>>>(d, seed, k, S, pf, mu, linv, X64, Z); break;
    case 10: qt::router_draw_kernel<10><<<nb, 256, 0, st>>>(d, seed, k, S, pf, mu, linv, X64, Z); break;
    case 12: qt::router_draw_kernel<12><<<nb, 256, 0, st>>>(d, seed, k, S, pf, mu, linv, X64, Z); break;
    default: qt::router_draw_kernel<16><<<nb, 256, 0, st>>>(d, seed, k, S, pf, mu, linv, X64, Z); break;
    }
    return cudaGetLastError();
}

int router_dm(int d)
{
    static const int dms[] = {2, 4, 6, 8, 10, 12, 16};
    for (int v : dms)
        if (v >= d) return v;
    return 0;
}

// Inverse of a lower-triangular matrix (FP64), zero matrix -> zero.
void tri_inverse(const double* L, int d, double* out)
{
    for (int e = 0; e < d * d; ++e) out[e] = 0.0;
    bool zero = true;
    for (int e = 0; e < d * d; ++e) zero = zero && L[e] == 0.0;
    if (zero) return;
    for (int c = 0; c < d; ++c) {
        out[c * d + c] = 1.0 / L[c * d + c];
        for (int r = c + 1; r < d; ++r) {
            double s = 0.0;
            for (int q = c; q < r; ++q) s += L[r * d + q] * out[q * d + c];
            out[r * d + c] = -s / L[r * d + r];
        }
    }
}

struct Arena {
    std::vector<void*> ptrs;
    ~Arena()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t get(T** out, size_t count)
    {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16));
        if (e == cudaSuccess) ptrs.push_back(p);
        *out = (T*)p;
        return e;
    }
};

}  // namespace

#define RT_CUDA(call)                          \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) {               \
            cudaGetLastError();                \
            qt_router_destroy(r);              \
            return e_ == cudaErrorMemoryAllocation ? QT_ENOMEM : QT_ECUDA; \
        }                                      \
    } while (0)

extern "C" qt_status qt_router_train(qt_ctx* ctx, const qt_model* model, const double* grids,
                                     const qt_router_config* cfg_in, uint64_t seed, qt_router** out, void* stream)
{
    if (!ctx || !model || !grids || !out) return QT_EINVAL;
    *out = nullptr;
    const int d = model->d, n = model->n;
    if (d < 1 || d > 16 || n < 1) return QT_EINVAL;
    const long long Nc = model->N[n];
    for (int k = 1; k <= n; ++k)
        if (model->N[k] != Nc) return QT_EUNSUPPORTED;
    if (Nc < kRtBuckets || Nc > 8192) return QT_EUNSUPPORTED;
    if (cfg_in && cfg_in->batch > 0 && cfg_in->batch < 64) return QT_EINVAL;
    qt_router_config cfg;
    memset(&cfg, 0, sizeof cfg);
    if (cfg_in) cfg = *cfg_in;
    const long long S = cfg.train_samples > 0 ? cfg.train_samples : 1000000;
    const int TL = std::min(n, cfg.train_layers > 0 ? cfg.train_layers : 8);
    const int epochs = cfg.epochs > 0 ? cfg.epochs : 8;
    const int Bt = cfg.batch > 0 ? cfg.batch : 4096;
    const int C = std::min<int>(cfg.neighbours > 0 ? cfg.neighbours : 1024, (int)Nc - 1);
    const float lr = cfg.lr > 0 ? cfg.lr : 3e-3f;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    const int dm = router_dm(d);

    qt_router* r = new (std::nothrow) qt_router();
    if (!r) return QT_ENOMEM;
    r->device = dev;
    r->d = d;
    r->n = n;
    r->N = (int)Nc;
    r->C = C;
    r->P = rt_param_count(d);
    std::vector<long long> off(n + 2, 0);
    for (int k = 0; k <= n; ++k) off[k + 1] = off[k] + model->N[k];
    const long long total_pts = off[n + 1];

    // ---- whitening matrices and centres (FP32, the centres of the screen's records)
    std::vector<float> linv((size_t)(n + 1) * d * d, 0.0f), mu((size_t)(n + 1) * d, 0.0f);
    std::vector<double> tmp((size_t)d * d);
    for (int k = 0; k <= n; ++k) {
        tri_inverse(model->L + (long long)k * d * d, d, tmp.data());
        for (int e = 0; e < d * d; ++e) linv[(size_t)k * d * d + e] = (float)tmp[e];
        for (int l = 0; l < d; ++l) mu[(size_t)k * d + l] = (float)model->m[(long long)k * d + l];
    }
    RT_CUDA(cudaMalloc(&r->linv, linv.size() * 4));
    RT_CUDA(cudaMemcpy(r->linv, linv.data(), linv.size() * 4, cudaMemcpyHostToDevice));

    // ---- buckets: k-means (64 centres) of the whitened points of the last grid
    std::vector<double> gl((size_t)Nc * d);
    RT_CUDA(cudaMemcpy(gl.data(), grids + off[n] * d, gl.size() * 8, cudaMemcpyDeviceToHost));
    std::vector<double> wz((size_t)Nc * d);
    {
        const double* Ln = model->L + (long long)n * d * d;
        tri_inverse(Ln, d, tmp.data());
        for (long long j = 0; j < Nc; ++j)
            for (int l = 0; l < d; ++l) {
                double a = 0.0;
                for (int q = 0; q <= l; ++q) a += tmp[l * d + q] * (gl[j * d + q] - model->m[(long long)n * d + q]);
                wz[j * d + l] = a;
            }
    }
    std::vector<double> cen((size_t)kRtBuckets * d);
    for (int b = 0; b < kRtBuckets; ++b)
        for (int l = 0; l < d; ++l) cen[b * d + l] = wz[(size_t)((long long)b * Nc / kRtBuckets) * d + l];
    std::vector<int> bucket_of((size_t)Nc, 0);
    for (int it = 0; it < 30; ++it) {
        for (long long j = 0; j < Nc; ++j) {
            double best = 1e300;
            int bi = 0;
            for (int b = 0; b < kRtBuckets; ++b) {
                double s = 0.0;
                for (int l = 0; l < d; ++l) {
                    const double t = wz[j * d + l] - cen[b * d + l];
                    s += t * t;
                }
                if (s < best) {
                    best = s;
                    bi = b;
                }
            }
            bucket_of[j] = bi;
        }
        std::vector<double> acc((size_t)kRtBuckets * d, 0.0);
        std::vector<long long> cnt(kRtBuckets, 0);
        for (long long j = 0; j < Nc; ++j) {
            ++cnt[bucket_of[j]];
            for (int l = 0; l < d; ++l) acc[bucket_of[j] * d + l] += wz[j * d + l];
        }
        for (int b = 0; b < kRtBuckets; ++b)
            if (cnt[b])
                for (int l = 0; l < d; ++l) cen[b * d + l] = acc[b * d + l] / cnt[b];
    }
    std::vector<int32_t> bstart(kRtBuckets + 1, 0), members((size_t)Nc);
    for (long long j = 0; j < Nc; ++j) ++bstart[bucket_of[j] + 1];
    for (int b = 0; b < kRtBuckets; ++b) bstart[b + 1] += bstart[b];
    {
        std::vector<int32_t> pos(bstart.begin(), bstart.end() - 1);
        for (long long j = 0; j < Nc; ++j) members[pos[bucket_of[j]]++] = (int32_t)j;
    }
    RT_CUDA(cudaMalloc(&r->bstart, bstart.size() * 4));
    RT_CUDA(cudaMalloc(&r->members, members.size() * 4));
    RT_CUDA(cudaMemcpy(r->bstart, bstart.data(), bstart.size() * 4, cudaMemcpyHostToDevice));
    RT_CUDA(cudaMemcpy(r->members, members.data(), members.size() * 4, cudaMemcpyHostToDevice));

    // ---- Elkan tables of grids 1..n
    const size_t tab = (size_t)(n + 1) * Nc * C;
    RT_CUDA(cudaMalloc(&r->nb_idx, tab * 4));
    RT_CUDA(cudaMalloc(&r->nb_dist, tab * 4));
    {
        int npow2 = 1;
        while (npow2 < Nc) npow2 <<= 1;
        const size_t sm = (size_t)npow2 * 8;
        RT_CUDA(cudaFuncSetAttribute(qt::elkan_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        dim3 grid((unsigned)Nc, (unsigned)n);   // grids 1..n, all of size Nc
        qt::elkan_table_kernel<<<grid, 256, sm, st>>>(grids, d, (int)Nc, C, npow2, off[1], r->nb_idx, r->nb_dist);
        RT_CUDA(cudaGetLastError());
    }

    // ---- checksum of the grids
    {
        unsigned long long* dck;
        RT_CUDA(cudaMalloc(&dck, 8));
        RT_CUDA(cudaMemsetAsync(dck, 0, 8, st));
        RT_CUDA(qt::launch_grid_checksum(grids, total_pts * d, dck, st));
        RT_CUDA(cudaMemcpyAsync(&r->checksum, dck, 8, cudaMemcpyDeviceToHost, st));
        RT_CUDA(cudaStreamSynchronize(st));
        cudaFree(dck);
    }

    // ---- parameters: seeded He initialisation (host), then training
    std::vector<float> P((size_t)r->P);
    {
        unsigned long long s = seed * 0x9E3779B97F4A7C15ull + 12345;
        auto nrm = [&]() {
            // Box-Muller on a 64-bit LCG (initialisation only)
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            const double u1 = ((s >> 11) + 0.5) * 0x1p-53;
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            const double u2 = ((s >> 11) + 0.5) * 0x1p-53;
            return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
        };
        size_t e = 0;
        for (int o = 0; o < kRtHidden * d; ++o) P[e++] = (float)(nrm() * std::sqrt(2.0 / d));
        for (int o = 0; o < kRtHidden; ++o) P[e++] = 0.0f;
        for (int o = 0; o < kRtHidden * kRtHidden; ++o) P[e++] = (float)(nrm() * std::sqrt(2.0 / kRtHidden));
        for (int o = 0; o < kRtHidden; ++o) P[e++] = 0.0f;
        for (int o = 0; o < kRtHidden * kRtBuckets; ++o) P[e++] = (float)(nrm() * std::sqrt(1.0 / kRtHidden));
        for (int o = 0; o < kRtBuckets; ++o) P[e++] = 0.0f;
    }
    RT_CUDA(cudaMalloc(&r->params, P.size() * 4));
    RT_CUDA(cudaMemcpy(r->params, P.data(), P.size() * 4, cudaMemcpyHostToDevice));

    double last_loss = 0.0, last_acc = 0.0;
    if (!cfg.untrained) {
        Arena ar;
        // training pairs from TL evenly spaced layers k in 1..n
        const long long Sk = (S + TL - 1) / TL;
        const long long Sall = Sk * TL;
        float* Z;
        int32_t* lab;
        double* X64;
        int32_t *cells, *cells2;
        uint32_t* cscr;
        float *pf, *dmu, *dli;
        int32_t* dbucket;
        RT_CUDA(ar.get(&Z, (size_t)Sall * d));
        RT_CUDA(ar.get(&lab, (size_t)Sall));
        RT_CUDA(ar.get(&X64, (size_t)Sk * d));
        RT_CUDA(ar.get(&cells, (size_t)Sk));
        RT_CUDA(ar.get(&cells2, (size_t)Sk));
        RT_CUDA(ar.get(&cscr, (size_t)Nc * Nc));
        RT_CUDA(ar.get(&pf, (size_t)param_count(d) + 4));
        RT_CUDA(ar.get(&dmu, (size_t)d));
        RT_CUDA(ar.get(&dli, (size_t)d * d));
        RT_CUDA(ar.get(&dbucket, (size_t)Nc));
        std::vector<int32_t> bo(bucket_of.begin(), bucket_of.end());
        RT_CUDA(cudaMemcpy(dbucket, bo.data(), bo.size() * 4, cudaMemcpyHostToDevice));
        qt_options o;
        qt_default_options(&o);
        o.form = QT_FORM_F32_RECHECK;
        o.counts_type = QT_COUNTS_U32;
        o.flags = QT_FLAG_NO_TUNE;
        for (int t = 0; t < TL; ++t) {
            const int k = 1 + (int)((long long)t * n / TL);
            std::vector<float> pk((size_t)param_count(d) + 4, 0.0f);
            for (int l = 0; l < d; ++l) pk[l] = (float)model->m[(long long)k * d + l];
            for (int e = 0; e < d * d; ++e) {
                const int rr = e / d, cc = e % d;
                pk[2 * d + e] = cc <= rr ? (float)model->L[(long long)k * d * d + e] : 0.0f;
            }
            RT_CUDA(cudaMemcpy(pf, pk.data(), pk.size() * 4, cudaMemcpyHostToDevice));
            RT_CUDA(cudaMemcpy(dmu, mu.data() + (size_t)k * d, (size_t)d * 4, cudaMemcpyHostToDevice));
            RT_CUDA(cudaMemcpy(dli, linv.data() + (size_t)k * d * d, (size_t)d * d * 4, cudaMemcpyHostToDevice));
            RT_CUDA(draw(dm, d, seed, k, Sk, pf, dmu, dli, X64, Z + (size_t)t * Sk * d, st));
            // exact cells of the draws with the library's own search
            const double* gk = grids + off[k] * d;
            qt_status qs = qt_counts_from_samples(ctx, d, gk, Nc, gk, Nc, X64, X64, Sk, &o, cscr, cells, cells2,
                                                  nullptr, stream);
            if (qs != QT_OK) {
                qt_router_destroy(r);
                return qs;
            }
            qt::gather_labels_kernel<<<(unsigned)((Sk + 255) / 256), 256, 0, st>>>(cells, dbucket, Sk,
                                                                                    lab + (size_t)t * Sk);
            RT_CUDA(cudaGetLastError());
        }
        // Adam on minibatches
        float *H1, *H2, *DL, *DH1, *DH2, *G, *Mm, *Vv;
        double* loss;
        int* correct;
        RT_CUDA(ar.get(&H1, (size_t)Bt * kRtHidden));
        RT_CUDA(ar.get(&H2, (size_t)Bt * kRtHidden));
        RT_CUDA(ar.get(&DL, (size_t)Bt * kRtBuckets));
        RT_CUDA(ar.get(&DH1, (size_t)Bt * kRtHidden));
        RT_CUDA(ar.get(&DH2, (size_t)Bt * kRtHidden));
        RT_CUDA(ar.get(&G, (size_t)r->P));
        RT_CUDA(ar.get(&Mm, (size_t)r->P));
        RT_CUDA(ar.get(&Vv, (size_t)r->P));
        RT_CUDA(ar.get(&loss, (size_t)Bt));
        RT_CUDA(ar.get(&correct, (size_t)Bt));
        RT_CUDA(cudaMemsetAsync(Mm, 0, (size_t)r->P * 4, st));
        RT_CUDA(cudaMemsetAsync(Vv, 0, (size_t)r->P * 4, st));
        // a fixed interleaving of the layers' pairs: batch j takes pairs j*Bt.. of a
        // permutation that strides across the layers
        const long long nbatch = Sall / Bt;
        std::vector<double> hl((size_t)Bt);
        std::vector<int> hc((size_t)Bt);
        long long step = 0;
        float* Zb;
        int32_t* Lb;
        RT_CUDA(ar.get(&Zb, (size_t)Bt * d));
        RT_CUDA(ar.get(&Lb, (size_t)Bt));
        for (int ep = 0; ep < epochs; ++ep) {
            double eloss = 0.0;
            long long ecorr = 0, ecount = 0;
            for (long long bi = 0; bi < nbatch; ++bi) {
                // batch bi: Bt / TL consecutive pairs from every training layer
                const long long per = Bt / TL;
                const long long rot = (bi + ep * 7919) % std::max<long long>(1, Sk / std::max<long long>(per, 1));
                for (int t = 0; t < TL; ++t) {
                    const long long src = (long long)t * Sk + rot * per;
                    const long long cnt = t == TL - 1 ? Bt - per * (TL - 1) : per;
                    RT_CUDA(cudaMemcpyAsync(Zb + (size_t)t * per * d, Z + (size_t)src * d, (size_t)cnt * d * 4,
                                            cudaMemcpyDeviceToDevice, st));
                    RT_CUDA(cudaMemcpyAsync(Lb + (size_t)t * per, lab + src, (size_t)cnt * 4,
                                            cudaMemcpyDeviceToDevice, st));
                }
                RT_CUDA(train_forward(dm, r->params, d, Zb, Lb, Bt, H1, H2, DL, loss, correct, st));
                qt::mlp_train_backward_kernel<<<(Bt + 127) / 128, 128, 0, st>>>(r->params, d, Bt, H1, H2, DL, DH1,
                                                                                 DH2);
                RT_CUDA(cudaGetLastError());
                qt::mlp_param_grad_kernel<<<(unsigned)((r->P + 255) / 256), 256, 0, st>>>(d, Bt, Zb, H1, H2, DL,
                                                                                           DH1, DH2, G);
                RT_CUDA(cudaGetLastError());
                ++step;
                qt::adam_kernel<<<(unsigned)((r->P + 255) / 256), 256, 0, st>>>(
                    (int)r->P, r->params, G, Mm, Vv, lr, (float)std::pow(0.9, (double)step),
                    (float)std::pow(0.999, (double)step));
                RT_CUDA(cudaGetLastError());
                if (ep == epochs - 1) {
                    RT_CUDA(cudaMemcpyAsync(hl.data(), loss, (size_t)Bt * 8, cudaMemcpyDeviceToHost, st));
                    RT_CUDA(cudaMemcpyAsync(hc.data(), correct, (size_t)Bt * 4, cudaMemcpyDeviceToHost, st));
                    RT_CUDA(cudaStreamSynchronize(st));
                    for (int b = 0; b < Bt; ++b) {
                        eloss += hl[b];
                        ecorr += hc[b];
                    }
                    ecount += Bt;
                }
            }
            if (ep == epochs - 1 && ecount) {
                last_loss = eloss / ecount;
                last_acc = (double)ecorr / ecount;
            }
        }
        RT_CUDA(cudaStreamSynchronize(st));
    }
    RT_CUDA(cudaStreamSynchronize(st));
    r->info.params = r->P;
    r->info.d = d;
    r->info.buckets = kRtBuckets;
    r->info.hidden = kRtHidden;
    r->info.neighbours = C;
    r->info.train_loss = last_loss;
    r->info.train_accuracy = last_acc;
    r->info.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = r;
    return QT_OK;
}

extern "C" qt_status qt_router_destroy(qt_router* r)
{
    if (!r) return QT_OK;
    cudaFree(r->params);
    cudaFree(r->linv);
    cudaFree(r->bstart);
    cudaFree(r->members);
    cudaFree(r->nb_idx);
    cudaFree(r->nb_dist);
    delete r;
    return QT_OK;
}

extern "C" qt_status qt_router_get_info(const qt_router* r, qt_router_info* info)
{
    if (!r || !info) return QT_EINVAL;
    *info = r->info;
    return QT_OK;
}

extern "C" qt_status qt_router_get_params(const qt_router* r, float* out, int64_t count)
{
    if (!r || !out || count != r->P) return QT_EINVAL;
    return cudaMemcpy(out, r->params, (size_t)count * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? QT_OK : QT_ECUDA;
}

extern "C" qt_status qt_router_set_params(qt_router* r, const float* in, int64_t count)
{
    if (!r || !in || count != r->P) return QT_EINVAL;
    return cudaMemcpy(r->params, in, (size_t)count * 4, cudaMemcpyHostToDevice) == cudaSuccess ? QT_OK : QT_ECUDA;
}

extern "C" qt_status qt_router_loss_grad(qt_ctx* ctx, const qt_router* rr, const float* z, const int32_t* labels,
                                         int64_t B, float* grad, double* loss_out, void* stream)
{
    if (!ctx || !rr || !z || !labels || !grad || !loss_out || B < 1 || B > (1 << 20)) return QT_EINVAL;
    qt_router* r = nullptr;   // RT_CUDA destroys r on failure: keep it null here
    cudaStream_t st = (cudaStream_t)stream;
    const int d = rr->d, dm = router_dm(d);
    Arena ar;
    float *H1, *H2, *DL, *DH1, *DH2;
    double* loss;
    int* correct;
    RT_CUDA(ar.get(&H1, (size_t)B * kRtHidden));
    RT_CUDA(ar.get(&H2, (size_t)B * kRtHidden));
    RT_CUDA(ar.get(&DL, (size_t)B * kRtBuckets));
    RT_CUDA(ar.get(&DH1, (size_t)B * kRtHidden));
    RT_CUDA(ar.get(&DH2, (size_t)B * kRtHidden));
    RT_CUDA(ar.get(&loss, (size_t)B));
    RT_CUDA(ar.get(&correct, (size_t)B));
    RT_CUDA(train_forward(dm, rr->params, d, z, labels, (int)B, H1, H2, DL, loss, correct, st));
    qt::mlp_train_backward_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(rr->params, d, (int)B, H1, H2, DL,
                                                                              DH1, DH2);
    RT_CUDA(cudaGetLastError());
    qt::mlp_param_grad_kernel<<<(unsigned)((rr->P + 255) / 256), 256, 0, st>>>(d, (int)B, z, H1, H2, DL, DH1, DH2,
                                                                               grad);
    RT_CUDA(cudaGetLastError());
    std::vector<double> hl((size_t)B);
    RT_CUDA(cudaMemcpyAsync(hl.data(), loss, (size_t)B * 8, cudaMemcpyDeviceToHost, st));
    RT_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : hl) s += v;
    *loss_out = s / (double)B;
    return QT_OK;
}
