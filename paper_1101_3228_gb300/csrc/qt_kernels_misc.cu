// qt_kernels_misc.cu -- small kernels around the forward step: preparation of
// the screened grid records, the backward induction of Sec. 2, the root price,
// and the sample-Lloyd (k-means) steps of the grid builder.
#include <cstdint>
#include <cuda_runtime.h>

#include "qt_internal.h"
#include "qt_sampler.cuh"

namespace qt {

// ------------------------------------------------------------------ grid records
//
// FP32 record of point c of grid g (centre mu_g, an FP32 vector):
//   [ fl32(|c - mu|^2 computed in FP64), fl32(c_0 - mu_0), ..., 0 ... ]
// padded rows (j >= N_g) carry cc = +inf so that they never win the screen.
// FP64 record: [c_0 .. c_{d-1}, 0 ...] (rec64 doubles).
// R_g = max_j |fl32(c_j - mu)| rounded up, accumulated with an integer max on
// the bits of a non-negative float.
__global__ void prep_records_kernel(const double* __restrict__ g64, GridInfo* gi, int ngrids, int d,
                                    int rec_floats, int rec64, long long total_recs, float* rec32,
                                    double* rec64out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total_recs) return;
    int lo = 0, hi = ngrids - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gi[mid].roff <= r) lo = mid; else hi = mid - 1;
    }
    const GridInfo& G = gi[lo];
    const long long j = r - G.roff;
    if (rec32) {
        float* out = rec32 + r * rec_floats;
        if (j < G.N) {
            const double* c = g64 + (G.goff + j) * d;
            double cc = 0.0, nr = 0.0;
            for (int l = 0; l < d; ++l) {
                const double t = c[l] - (double)G.mu[l];
                cc += t * t;
                const float tf = __double2float_rn(t);
                out[1 + l] = tf;
                nr += (double)tf * (double)tf;
            }
            for (int l = d + 1; l < rec_floats; ++l) out[l] = 0.0f;
            out[0] = __double2float_rn(cc);
            const float R = __double2float_ru(sqrt(nr) * (1.0 + 0x1p-50));
            atomicMax(reinterpret_cast<unsigned int*>(&gi[lo].R), __float_as_uint(R));
        } else {
            out[0] = __int_as_float(0x7F800000);
            for (int l = 1; l < rec_floats; ++l) out[l] = 0.0f;
        }
    }
    if (rec64out) {
        double* out = rec64out + r * rec64;
        if (j < G.N) {
            const double* c = g64 + (G.goff + j) * d;
            for (int l = 0; l < d; ++l) out[l] = c[l];
            for (int l = d; l < rec64; ++l) out[l] = 0.0;
        } else {
            for (int l = 0; l < rec64; ++l) out[l] = __longlong_as_double(0x7FF0000000000000LL);
        }
    }
}

// ------------------------------------------------------------------ backward induction
//
// V_k(i) = max(phi_k(i), (sum_j p_ij V_{k+1}(j)) / p_i), p_i = sum_j p_ij; empty
// rows keep phi_k(i).  One warp per row: lane l sums j = l, l+32, ... in
// ascending order (products and sums rounded one at a time), then a butterfly
// over offsets 16, 8, 4, 2, 1 combines the lanes, so every run gives the same
// bits.
__global__ void backward_layer_kernel(const void* __restrict__ counts, int u32, long long coff, int Nk, int Nk1,
                                      const double* __restrict__ phik, const double* __restrict__ Vnext,
                                      double* __restrict__ Vk)
{
    const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= Nk) return;
    const long long row = coff + (long long)warp * Nk1;
    double acc = 0.0;
    long long ci = 0;
    if (u32) {
        const uint32_t* c = reinterpret_cast<const uint32_t*>(counts) + row;
        for (int j = lane; j < Nk1; j += 32) {
            const uint32_t v = c[j];
            ci += v;
            acc = __dadd_rn(acc, __dmul_rn((double)v, Vnext[j]));
        }
    } else {
        const long long* c = reinterpret_cast<const long long*>(counts) + row;
        for (int j = lane; j < Nk1; j += 32) {
            const long long v = c[j];
            ci += v;
            acc = __dadd_rn(acc, __dmul_rn((double)v, Vnext[j]));
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, off));
        ci += __shfl_xor_sync(0xFFFFFFFFu, ci, off);
    }
    if (lane == 0) {
        const double ph = phik[warp];
        if (ci == 0) {
            Vk[warp] = ph;
        } else {
            const double cont = __ddiv_rn(acc, (double)ci);
            Vk[warp] = ph > cont ? ph : cont;
        }
    }
}

// ------------------------------------------------------------------ swing option
//
// Eq. (stochCtrl) with the bang-bang BDP of Sec. 2: controls x in {0, 1} at
// dates k = 0..n-1, consumption state Q, chi(Q, x) = Q + x, x admissible at
// (k, Q) when F(k+1, Q + x), F(k, Q) = (Q <= Qmax and Q + n - k >= Qmin):
//   P_k(i, Q) = max over admissible x of x v_k(i) + C_k(i, Q + x),
//   C_k(i, Q') = (sum_j p^k_ij P_{k+1}(j, Q')) / p^k_i   (0 for an empty row),
// -inf where no x is admissible.  P blocks are Q-major: [Qmax + 1][N].  One
// warp per (row i, chunk of kSwingQ consumption states) walks its Q upwards and
// carries C(i, Q + 1) to the next Q; every continuation is summed by one warp
// in the order of backward_layer_kernel (lanes j mod 32 ascending, then the
// fixed butterfly), whichever warp it is, which makes the one-right swing
// (Qmax = 1) the Bermudan of qt_backward bit for bit.
__device__ __forceinline__ bool swing_feasible(int n, int k, int Q, int Qmin, int Qmax)
{
    return Q <= Qmax && Q + (n - k) >= Qmin;
}

__global__ void swing_terminal_kernel(int Nn, int n, int Qmin, int Qmax, double* __restrict__ Pn)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)(Qmax + 1) * Nn) return;
    const int Q = (int)(e / Nn);
    Pn[e] = swing_feasible(n, n, Q, Qmin, Qmax) ? 0.0 : __longlong_as_double(0xFFF0000000000000LL);
}

__global__ void swing_layer_kernel(const void* __restrict__ counts, int u32, long long coff, int Nk, int Nk1,
                                   const double* __restrict__ vk, const double* __restrict__ Pnext,
                                   double* __restrict__ Pk, int n, int k, int Qmin, int Qmax)
{
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int qchunks = (Qmax + kSwingQ) / kSwingQ;
    if (gw >= (long long)Nk * qchunks) return;
    const int warp = (int)(gw / qchunks);              // grid row i
    const int q0 = (int)(gw % qchunks) * kSwingQ;      // first consumption state of this warp
    const long long row = coff + (long long)warp * Nk1;
    const uint32_t* c32 = reinterpret_cast<const uint32_t*>(counts) + row;
    const long long* c64 = reinterpret_cast<const long long*>(counts) + row;
    long long ci = 0;
    for (int j = lane; j < Nk1; j += 32) ci += u32 ? (long long)c32[j] : c64[j];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) ci += __shfl_xor_sync(0xFFFFFFFFu, ci, off);
    const double ninf = __longlong_as_double(0xFFF0000000000000LL);
    // continuation C(i, Q') for a feasible Q' at date k + 1
    auto cont = [&](int Qp) -> double {
        if (!swing_feasible(n, k + 1, Qp, Qmin, Qmax)) return ninf;
        const double* Pq = Pnext + (long long)Qp * Nk1;
        double acc = 0.0;
        for (int j = lane; j < Nk1; j += 32) {
            const double cv = u32 ? (double)c32[j] : (double)c64[j];
            acc = __dadd_rn(acc, __dmul_rn(cv, Pq[j]));
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, off));
        return ci == 0 ? 0.0 : __ddiv_rn(acc, (double)ci);
    };
    const double v = vk[warp];
    double c_cur = cont(q0);
    const int q1 = min(Qmax, q0 + kSwingQ - 1);
    for (int Q = q0; Q <= q1; ++Q) {
        const double c_next = Q + 1 <= Qmax ? cont(Q + 1) : ninf;
        double best = ninf;
        if (swing_feasible(n, k + 1, Q, Qmin, Qmax)) best = c_cur;                  // x = 0
        if (swing_feasible(n, k + 1, Q + 1, Qmin, Qmax)) {                          // x = 1
            const double val = __dadd_rn(v, c_next);
            if (val > best) best = val;
        }
        if (lane == 0) Pk[(long long)Q * Nk + warp] = best;
        c_cur = c_next;
    }
}

// Status of one launch folded into an accumulator (the fused price mode runs
// one launch per layer pair, each clearing its own status block): the first
// error code and site are kept, the counters are summed.  One thread.
__global__ void fold_status_kernel(const DevStatus* __restrict__ src, DevStatus* acc)
{
    if (acc->code == 0 && src->code != 0) {
        acc->code = src->code;
        acc->where = src->where;
    }
    acc->rechecks += src->rechecks;
    acc->candidates += src->candidates;
    acc->done_items += src->done_items;
    acc->spare[0] = src->spare[0];
    for (int q = 1; q < 4; ++q) acc->spare[q] += src->spare[q];
}

// Root value: sum_i (p^0_i / M) V_0(i), one warp, same fixed order as above.
__global__ void root_price_kernel(const void* __restrict__ counts, int u32, int N0, int N1,
                                  const double* __restrict__ V0, double* out)
{
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    long long tot = 0;
    for (int i = lane; i < N0; i += 32) {
        long long ci = 0;
        for (int j = 0; j < N1; ++j)
            ci += u32 ? (long long)reinterpret_cast<const uint32_t*>(counts)[(long long)i * N1 + j]
                      : reinterpret_cast<const long long*>(counts)[(long long)i * N1 + j];
        tot += ci;
        acc = __dadd_rn(acc, __dmul_rn((double)ci, V0[i]));
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, off));
        tot += __shfl_xor_sync(0xFFFFFFFFu, tot, off);
    }
    if (lane == 0) *out = tot > 0 ? __ddiv_rn(acc, (double)tot) : 0.0;
}

// ------------------------------------------------------------------ sample Lloyd (grid builder)

// Seeded N(0, I_d) training draws from the same Philox/Box-Muller sampler
// (layer index 0xFFFF separates this stream from the forward step's).
__global__ void kmeans_draw_kernel(int d, unsigned long long seed, long long S, float* Z)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S) return;
    float g[kDMax];
    normals_f32<kDMax>(seed, 0xFFFF, (unsigned long long)t, d, g);
    for (int l = 0; l < d; ++l) Z[t * d + l] = g[l];
}

// Nearest centre in FP32 (training assignment; exactness is not needed here)
// and fixed-point sums (scale 2^36) so that the centroids do not depend on the
// order of the atomics.
__global__ void kmeans_assign_kernel(int d, long long S, const float* __restrict__ Z, int N,
                                     const float* __restrict__ C, unsigned long long* sums,
                                     unsigned long long* cnt, int use_smem)
{
    extern __shared__ float sC_dyn[];
    if (use_smem) {
        for (int e = threadIdx.x; e < N * d; e += blockDim.x) sC_dyn[e] = C[e];
        __syncthreads();
    }
    const float* sC = use_smem ? sC_dyn : C;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S) return;
    float z[kDMax];
    for (int l = 0; l < d; ++l) z[l] = Z[t * d + l];
    float best = __int_as_float(0x7F800000);
    int bi = 0;
    for (int j = 0; j < N; ++j) {
        float acc = 0.f;
        for (int l = 0; l < d; ++l) {
            const float df = z[l] - sC[j * d + l];
            acc = fmaf(df, df, acc);
        }
        if (acc < best) {
            best = acc;
            bi = j;
        }
    }
    atomicAdd(&cnt[bi], 1ull);
    for (int l = 0; l < d; ++l) {
        const long long q = __double2ll_rn((double)z[l] * 68719476736.0);
        atomicAdd(&sums[(long long)bi * d + l], (unsigned long long)q);
    }
}

__global__ void kmeans_update_kernel(int d, int N, const unsigned long long* sums, const unsigned long long* cnt,
                                     float* C)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const unsigned long long c = cnt[j];
    if (c == 0) return;  // empty cell keeps its centre
    for (int l = 0; l < d; ++l) {
        const long long s = (long long)sums[(long long)j * d + l];
        C[j * d + l] = (float)(((double)s / 68719476736.0) / (double)c);
    }
}

// Layer grids from a base grid: x = m_k + L_k g.
__global__ void map_grid_kernel(int d, int N, const double* __restrict__ G, const double* __restrict__ mk,
                                const double* __restrict__ Lk, double* out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    for (int l = 0; l < d; ++l) {
        double acc = mk[l];
        for (int q = 0; q <= l; ++q) acc += Lk[l * d + q] * G[j * d + q];
        out[(long long)j * d + l] = acc;
    }
}

}  // namespace qt
