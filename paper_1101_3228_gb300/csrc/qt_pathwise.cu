// qt_pathwise.cu -- Algorithm II of Pages & Wilbertz (arXiv:1101.3228, Sec. 3):
// the path-wise estimator of the transition counts.  Each path is simulated
// through every layer, X_{k+1} = b_k + A_k X_k + S_k(X_k) T_k eps_k, and each
// layer costs ONE nearest-cell search (Algorithm III spends two, because it
// draws every layer's pair afresh); p^k_ij counts consecutive cells i -> j.
//
// S_k = I is the AR(1) chain of Prop. 1.  The Euler-scheme chain scales row l
// of the innovation by s_l = sqrt(max(alpha_l + beta_l x_l, 0)): the Euler step
// of a square-root diffusion.  Such a chain is not AR(1), so its layers cannot
// be drawn independently and Algorithm III does not apply to it; the path-wise
// simulation does.
//
// Sampler: X_0 = m_0 + L_0 z with z = normals [0, d) of stream (m, layer 0);
// eps_k = normals [d, 2d) of stream (m, k) -- so the first step is exactly
// Algorithm III's layer-0 pair.  Each operation is rounded in the order
//   s_l = sqrt(max(alpha_l + beta_l * x_l, 0)); t_lq = s_l * T_lq;
//   acc = b_l; acc += A_lq * x_q (q = 0..d-1); acc += t_lq * eps_q (q = 0..l)
// in the sample precision (with the AR(1) chain t_lq = T_lq).
//
// GB300 layout: one persistent kernel; a work item is a tile of paths
// (256 threads x S paths), handed out by an L2 atomic counter.  A CTA carries
// its tile through all layers.  The FP32 records of the grids go through two
// shared-memory buffers as a sequence of segments (a whole grid per segment
// when it fits half the shared memory, else several): while the CTA screens one
// segment, the bulk copy (TMA engine) of the next is in flight.  The search is
// the FP32 screen with its certificate and the exact window search of the
// Algorithm III kernel (qt_forward.cuh), so every cell is the exact FP64 cell
// of the library contract.  Counts go to L2 with red.global.add (every CTA touches every
// layer, so a private histogram would be flushed n times per tile).
#include "qt_forward.cuh"
#include "qt_launch.h"

namespace qt {

namespace {

// Normals [lo, hi) of stream (m, k), FP32: only the Box-Muller pairs that
// overlap the range are evaluated (each Philox call yields two pairs).
template <int CNT>
__device__ __forceinline__ void normals_range_f32(uint64_t seed, int k, uint64_t m, int lo, int hi, float (&g)[CNT])
{
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const uint32_t m0 = (uint32_t)m, m1 = (uint32_t)(m >> 32);
#pragma unroll
    for (int r = 0; r < (CNT + 3) / 4; ++r) {
        if (4 * r + 4 > lo && 4 * r < hi) {
            const Philox4 w = philox4x32_10(m0, m1, (uint32_t)k, (uint32_t)r, key0, key1);
#pragma unroll
            for (int pair = 0; pair < 2; ++pair) {
                const int q = 4 * r + 2 * pair;
                if (q + 2 > lo && q < hi) {
                    const float u0 = uniform_f32(w.v[2 * pair]);
                    const float u1 = uniform_f32(w.v[2 * pair + 1]);
                    const float rad = __fsqrt_rn(__fmul_rn(-2.0f, ln_f32(u0)));
                    float sn, cs;
                    sincos2pi_f32(u1, sn, cs);
                    if (q < CNT) g[q] = __fmul_rn(rad, cs);
                    if (q + 1 < CNT) g[q + 1] = __fmul_rn(rad, sn);
                }
            }
        }
    }
}

template <int CNT>
__device__ __forceinline__ void normals_range_f64(uint64_t seed, int k, uint64_t m, int lo, int hi, double (&g)[CNT])
{
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const uint32_t m0 = (uint32_t)m, m1 = (uint32_t)(m >> 32);
#pragma unroll
    for (int r = 0; r < (CNT + 1) / 2; ++r) {
        if (2 * r + 2 > lo && 2 * r < hi) {
            const Philox4 w = philox4x32_10(m0, m1, (uint32_t)k, (uint32_t)r, key0, key1);
            const double u0 = uniform_f64(w.v[0], w.v[1]);
            const double u1 = uniform_f64(w.v[2], w.v[3]);
            const double rad = __dsqrt_rn(__dmul_rn(-2.0, ln_f64(u0)));
            double sn, cs;
            sincos2pi_f64(u1, sn, cs);
            if (2 * r < CNT) g[2 * r] = __dmul_rn(rad, cs);
            if (2 * r + 1 < CNT) g[2 * r + 1] = __dmul_rn(rad, sn);
        }
    }
}

// Layer parameters as packed by the host (param_stride): m[d], b[d], L[d*d],
// A[d*d], T[d*d], alpha[d], beta[d].

// X_0 = m_0 + L_0 z (stored in X, sample precision T).
template <int DM>
__device__ __forceinline__ void path_start_f32(const float* __restrict__ P, int d, uint64_t seed, uint64_t m,
                                               float (&X)[DM])
{
    float g[2 * DM];
    normals_range_f32<2 * DM>(seed, 0, m, 0, d, g);
    const float* pm = P;
    const float* pL = P + 2 * d;
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        float acc = 0.0f;
        if (l < d) {
            acc = pm[l];
#pragma unroll
            for (int q = 0; q <= l; ++q) acc = __fadd_rn(acc, __fmul_rn(pL[l * d + q], g[q]));
        }
        X[l] = acc;
    }
}

template <int DM>
__device__ __forceinline__ void path_start_f64(const double* __restrict__ P, int d, uint64_t seed, uint64_t m,
                                               double (&X)[DM])
{
    double g[2 * DM];
    normals_range_f64<2 * DM>(seed, 0, m, 0, d, g);
    const double* pm = P;
    const double* pL = P + 2 * d;
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        double acc = 0.0;
        if (l < d) {
            acc = pm[l];
#pragma unroll
            for (int q = 0; q <= l; ++q) acc = __dadd_rn(acc, __dmul_rn(pL[l * d + q], g[q]));
        }
        X[l] = acc;
    }
}

// One step of the chain at layer k (parameters P of layer k).
template <int DM>
__device__ __forceinline__ void path_step_f32(const float* __restrict__ P, int d, bool euler, uint64_t seed, int k,
                                              uint64_t m, float (&X)[DM])
{
    float g[2 * DM];
    normals_range_f32<2 * DM>(seed, k, m, d, 2 * d, g);
    const float* pb = P + d;
    const float* pA = P + 2 * d + d * d;
    const float* pT = pA + d * d;
    const float* pal = pT + d * d;
    const float* pbe = pal + d;
    float sc[DM], Xn[DM];
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        sc[l] = 1.0f;
        if (euler && l < d) {
            const float u = __fadd_rn(pal[l], __fmul_rn(pbe[l], X[l]));
            sc[l] = __fsqrt_rn(u > 0.0f ? u : 0.0f);
        }
    }
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        float acc = 0.0f;
        if (l < d) {
            acc = pb[l];
#pragma unroll
            for (int q = 0; q < DM; ++q)
                if (q < d) acc = __fadd_rn(acc, __fmul_rn(pA[l * d + q], X[q]));
#pragma unroll
            for (int q = 0; q <= l; ++q) {
                const float t = euler ? __fmul_rn(sc[l], pT[l * d + q]) : pT[l * d + q];
                acc = __fadd_rn(acc, __fmul_rn(t, g[d + q]));
            }
        }
        Xn[l] = acc;
    }
#pragma unroll
    for (int l = 0; l < DM; ++l) X[l] = Xn[l];
}

template <int DM>
__device__ __forceinline__ void path_step_f64(const double* __restrict__ P, int d, bool euler, uint64_t seed, int k,
                                              uint64_t m, double (&X)[DM])
{
    double g[2 * DM];
    normals_range_f64<2 * DM>(seed, k, m, d, 2 * d, g);
    const double* pb = P + d;
    const double* pA = P + 2 * d + d * d;
    const double* pT = pA + d * d;
    const double* pal = pT + d * d;
    const double* pbe = pal + d;
    double sc[DM], Xn[DM];
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        sc[l] = 1.0;
        if (euler && l < d) {
            const double u = __dadd_rn(pal[l], __dmul_rn(pbe[l], X[l]));
            sc[l] = __dsqrt_rn(u > 0.0 ? u : 0.0);
        }
    }
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        double acc = 0.0;
        if (l < d) {
            acc = pb[l];
#pragma unroll
            for (int q = 0; q < DM; ++q)
                if (q < d) acc = __dadd_rn(acc, __dmul_rn(pA[l * d + q], X[q]));
#pragma unroll
            for (int q = 0; q <= l; ++q) {
                const double t = euler ? __dmul_rn(sc[l], pT[l * d + q]) : pT[l * d + q];
                acc = __dadd_rn(acc, __dmul_rn(t, g[d + q]));
            }
        }
        Xn[l] = acc;
    }
#pragma unroll
    for (int l = 0; l < DM; ++l) X[l] = Xn[l];
}

template <bool F32>
struct SampleType {
    using T = double;
};
template <>
struct SampleType<true> {
    using T = float;
};

}  // namespace

template <int DM, int S, bool F32, bool STREAMED>
__global__ void __launch_bounds__(256, (DM <= 4 ? 2 : 1)) pathwise_kernel(const ForwardParams p)
{
    using T = typename SampleType<F32>::T;
    constexpr int F = Rec32<DM>::kFloats;
    extern __shared__ __align__(128) unsigned char dsm_pw[];
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ long long s_item;
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int d = p.d;
    const int n = p.n;
    const int seg = p.seg_records;                       // records per segment, a multiple of kChunk
    const uint32_t buf_bytes = (uint32_t)p.smem_grid_bytes / 2u;
    const bool euler = p.pathwise_euler != 0;

    if (tid == 0) {
        mbar_init(smem_u32(&s_bar[0]), 1);
        mbar_init(smem_u32(&s_bar[1]), 1);
        fence_proxy_async();
        s_abort = 0;
    }
    __syncthreads();
    // the segment sequence of an item: grids 0..n in order, each in ceil(Npad / seg)
    // segments; segment number c of the sequence goes to buffer c & 1
    auto nseg = [&](int g) { return (p.grids[g].Npad + seg - 1) / seg; };
    long long total_segs = 0;
    for (int g = 0; g <= n; ++g) total_segs += nseg(g);
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    int sg = 0, st_seg = 0;                              // staging cursor (thread 0)

    // bulk copy of the next segment of the sequence into buffer c & 1 (thread 0)
    auto stage_next = [&](long long c) {
        const GridInfo& G = p.grids[sg];
        const int first = st_seg * seg;
        const int cnt = min(seg, G.Npad - first);
        const uint32_t bytes = (uint32_t)cnt * F * 4u;
        const uint32_t bar = smem_u32(&s_bar[c & 1]);
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(smem_u32(dsm_pw + (c & 1) * buf_bytes), p.rec32 + (G.roff + first) * F, bytes, bar);
        if (++st_seg == nseg(sg)) {
            st_seg = 0;
            ++sg;
        }
    };

    while (true) {
        if (tid == 0) {
            long long it = -1;
            if (*((volatile int32_t*)&p.status->code) == 0) it = (long long)atomicAdd(&p.status->queue, 1ull);
            s_item = it;
            if (it >= 0 && it < p.total_items) {
                sg = 0;
                st_seg = 0;
                stage_next(0);
                if (total_segs > 1) stage_next(1);
            }
        }
        __syncthreads();
        const long long item = s_item;
        if (item < 0 || item >= p.total_items) break;
        pending[0] = true;
        pending[1] = total_segs > 1;

        const unsigned long long mtile = (unsigned long long)item * (unsigned long long)p.tile;
        unsigned long long ms[S];
        bool valid[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            ms[s] = mtile + (unsigned long long)(s * blockDim.x + tid);
            valid[s] = ms[s] < p.M;
        }
        T x[S][DM];       // path states in the sample precision
        int cell[S];
        // ---- start states X_0
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const unsigned long long m = valid[s] ? ms[s] : mtile;
            if constexpr (F32) path_start_f32<DM>(p.params_f, d, p.seed, m, x[s]);
            else path_start_f64<DM>(p.params_d, d, p.seed, m, x[s]);
        }
        bool aborted = false;
        long long cur = 0;                               // next segment of the sequence to scan
        // ---- g = 0: the cell of X_0; g = k + 1: step k, then the cell of X_{k+1}
        for (int g = 0; g <= n && !aborted; ++g) {
            const int k = g - 1;
            if (k >= 0) {
                const float* gpf = p.params_f + (long long)k * p.params_stride;
                const double* gpd = p.params_d + (long long)k * p.params_stride;
                // dump row k: X_k before the step
                if (p.dump_count > 0) {
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        if (!valid[s] || (ms[s] % (unsigned long long)p.dump_stride) != 0ull) continue;
                        const unsigned long long t = ms[s] / (unsigned long long)p.dump_stride;
                        if (t >= (unsigned long long)p.dump_count) continue;
                        const long long row = (long long)k * p.dump_count + (long long)t;
                        for (int l = 0; l < d; ++l) p.dumpX[row * d + l] = (double)x[s][l];
                    }
                }
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const unsigned long long m = valid[s] ? ms[s] : mtile;
                    if constexpr (F32) path_step_f32<DM>(gpf, d, euler, p.seed, k, m, x[s]);
                    else path_step_f64<DM>(gpd, d, euler, p.seed, k, m, x[s]);
                }
            }
            const GridInfo& G = p.grids[g];
            // ---- centre on Gamma_g
            float xa[S][DM], Aa[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                float na = 0.f;
#pragma unroll
                for (int l = 0; l < DM; ++l) {
                    float ax = 0.0f;
                    if (l < d) {
                        if constexpr (F32) ax = __fsub_rn(x[s][l], G.mu[l]);
                        else ax = __double2float_rn(__dsub_rn(x[s][l], (double)G.mu[l]));
                    }
                    na = __fmaf_rn(ax, ax, na);
                    xa[s][l] = -2.0f * ax;
                }
                Aa[s] = __fsqrt_rn(na);
            }
            // ---- FP32 screen over the grid's segments; the best chunk is resolved
            // while its segment is in shared memory (a grid in one segment: after
            // the scan, with no resolution state live across it)
            ScanState<S> st;
            ResolveState<S> rs;
            scan_init<S>(st);
            resolve_init<S>(rs);
            const int Npad = G.Npad;
            const int ns = nseg(g);
            int cj[S];
            bool need[S];
            if (!STREAMED) {    // every grid is one segment
                const int b = (int)(cur & 1);
                if (!mbar_wait_bounded(smem_u32(&s_bar[b]), phase[b], p.spin_budget)) {
                    record_error(p.status, 4 /* QT_ETIMEOUT */, 40);
                    s_abort = 1;
                    mbar_wait_bounded(smem_u32(&s_bar[b]), phase[b], kDrainUs);
                }
                phase[b] ^= 1u;
                pending[b] = false;
                __syncthreads();
                if (s_abort) break;
                const float* rec = reinterpret_cast<const float*>(dsm_pw + b * buf_bytes);
                screen_scan<DM, S>(rec, Npad / kChunk, 0, xa, st);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    int idx;
                    float S1, r1;
                    resolve_one<DM>(rec, st.bc[s], xa[s], st.B1[s], idx, S1, r1);
                    const float second = fminf(st.B2[s], S1);
                    const bool cert = idx >= 0 && screen_certified(d, Aa[s], st.B1[s], second, r1);
                    cj[s] = idx;
                    need[s] = !cert && valid[s];
                }
                __syncthreads();   // every warp is done with buffer b
                if (cur + 2 < total_segs) {
                    if (tid == 0) stage_next(cur + 2);
                    pending[b] = true;
                }
                ++cur;
            }
            for (int t = 0; STREAMED && t < ns; ++t) {
                const int b = (int)(cur & 1);
                if (!mbar_wait_bounded(smem_u32(&s_bar[b]), phase[b], p.spin_budget)) {
                    // give up: raise the CTA's abort flag (read by every thread after
                    // the barrier) and let the copy land
                    record_error(p.status, 4 /* QT_ETIMEOUT */, 40);
                    s_abort = 1;
                    mbar_wait_bounded(smem_u32(&s_bar[b]), phase[b], kDrainUs);
                }
                phase[b] ^= 1u;
                pending[b] = false;
                __syncthreads();
                if (s_abort) {
                    aborted = true;
                    break;
                }
                const float* rec = reinterpret_cast<const float*>(dsm_pw + b * buf_bytes);
                const int cnt = min(seg, Npad - t * seg);
                const int c0 = t * seg / kChunk;
                screen_scan<DM, S>(rec, cnt / kChunk, c0, xa, st);
                screen_resolve<DM, S>(rec, cnt / kChunk, c0, xa, st, rs);
                __syncthreads();   // every warp is done with buffer b
                if (cur + 2 < total_segs) {
                    if (tid == 0) stage_next(cur + 2);
                    pending[b] = true;
                }
                ++cur;
            }
            if (aborted) break;
            if (STREAMED) {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const float second = fminf(st.B2[s], rs.S1[s]);
                    const bool cert = rs.idx[s] >= 0 && screen_certified(d, Aa[s], st.B1[s], second, rs.r1[s]);
                    cj[s] = rs.idx[s];
                    need[s] = !cert && valid[s];
                }
            }
            // ---- exact window search of the uncertified, one warp per search (records from L2)
            const float* grec = p.rec32 + G.roff * F;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                unsigned mask = __ballot_sync(0xFFFFFFFFu, need[s]);
                if (mask == 0) continue;
                double z[DM];
#pragma unroll
                for (int l = 0; l < DM; ++l) z[l] = (l < d) ? (double)x[s][l] : 0.0;
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int r = warp_window_nn<DM>(xa[s], Aa[s], z, src, grec, Npad, p.g64 + G.goff * d, G.N, d);
                    if (lane == src) cj[s] = r;
                    if (lane == 0) atomicAdd(&p.status->rechecks, 1ull);
                }
            }
            // ---- counters p^k_ij over consecutive cells, dumps
#pragma unroll
            for (int s = 0; s < S; ++s) {
                if (!valid[s]) {
                    cell[s] = 0;
                    continue;
                }
                const int j = cj[s];
                if ((unsigned)j >= (unsigned)G.N) {
                    record_error(p.status, 6 /* QT_EDEVICE */, 41);
                    cell[s] = 0;
                    continue;
                }
                if (k >= 0) {
                    const LayerDesc& L = p.layers[k];
                    const int i = cell[s];
                    count_add(p.counts, p.counts_u32, L.coff + (long long)i * L.NB + j, 1u);
                    if (p.dump_count > 0 && (ms[s] % (unsigned long long)p.dump_stride) == 0ull) {
                        const unsigned long long t = ms[s] / (unsigned long long)p.dump_stride;
                        if (t < (unsigned long long)p.dump_count) {
                            const long long row = (long long)k * p.dump_count + (long long)t;
                            for (int l = 0; l < d; ++l) p.dumpY[row * d + l] = (double)x[s][l];
                            p.dumpI[row] = i;
                            p.dumpJ[row] = j;
                        }
                    }
                }
                cell[s] = j;
            }
        }
        if (aborted) {
            // let the copies still in flight land before the CTA leaves
            for (int b = 0; b < 2; ++b)
                if (pending[b]) mbar_wait_bounded(smem_u32(&s_bar[b]), phase[b], kDrainUs);
            break;
        }
    }
}

template <int DM, int S, bool F32, bool STREAMED>
static cudaError_t launch_pw(const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st)
{
    auto kern = pathwise_kernel<DM, S, F32, STREAMED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, dyn);
    if (e != cudaSuccess) return e;
    if (b < 1) return cudaErrorInvalidConfiguration;
    *bps = b;
    long long grid = (long long)num_sms * b;
    if (grid > p.total_items) grid = p.total_items;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 256, dyn, st>>>(p);
    return cudaGetLastError();
}

// Compiled (dimension class, paths per thread) pairs: grids resident in one
// segment each (FP32 samples for every class, FP64 samples for the small
// classes), and grids streamed in several segments (one choice per class).
static const int kPwF32[][2] = {{1, 8}, {1, 2}, {2, 8}, {2, 4}, {2, 2}, {2, 1}, {3, 4}, {4, 4}, {4, 1},
                                {6, 2}, {8, 2}, {8, 1}, {10, 2}, {10, 1}, {12, 1}, {16, 1}};
static const int kPwF64[][2] = {{1, 4}, {1, 1}, {2, 4}, {2, 1}, {4, 2}, {8, 1}};
static const int kPwStreamF32[][2] = {{1, 4}, {2, 4}, {3, 4}, {4, 4}, {6, 2}, {8, 2}, {10, 2}, {12, 1}, {16, 1}};
static const int kPwStreamF64[][2] = {{1, 2}, {2, 2}, {4, 1}, {8, 1}};

bool pathwise_variant_exists(int dm, int S, bool f32, bool streamed)
{
    auto in = [&](const int (*tab)[2], int count) {
        for (int i = 0; i < count; ++i)
            if (tab[i][0] == dm && tab[i][1] == S) return true;
        return false;
    };
    if (streamed)
        return f32 ? in(kPwStreamF32, (int)(sizeof kPwStreamF32 / sizeof kPwStreamF32[0]))
                   : in(kPwStreamF64, (int)(sizeof kPwStreamF64 / sizeof kPwStreamF64[0]));
    return f32 ? in(kPwF32, (int)(sizeof kPwF32 / sizeof kPwF32[0]))
               : in(kPwF64, (int)(sizeof kPwF64 / sizeof kPwF64[0]));
}

// Paths per thread: the register-budget choice (the compiled one when the grids
// are streamed), lowered while the path tiles would not give every CTA slot
// (ctas = SMs x resident CTAs) about two tiles -- the path-wise form has only
// M paths of parallelism.
int pathwise_default_spt(int dm, bool f32, bool streamed, long long M, long long ctas)
{
    int S;
    if (streamed) {
        S = 1;
        for (int c : {4, 2, 1})
            if (pathwise_variant_exists(dm, c, f32, true)) {
                S = c;
                break;
            }
        return S;
    }
    S = f32 ? (dm <= 2 ? 8 : (dm <= 4 ? 4 : (dm <= 10 ? 2 : 1))) : (dm <= 2 ? 4 : (dm <= 4 ? 2 : 1));
    while (S > 1) {
        const int next = S / 2;
        if (M >= 2ll * ctas * 256 * S || !pathwise_variant_exists(dm, next, f32, false)) break;
        S = next;
    }
    return S;
}

cudaError_t launch_pathwise(int dm, int S, bool f32, bool streamed, const ForwardParams& p, int dyn, int num_sms,
                            int* bps, cudaStream_t st)
{
#define QT_CASE(D, SS, F, ST) \
    if (dm == D && S == SS && f32 == F && streamed == ST) return launch_pw<D, SS, F, ST>(p, dyn, num_sms, bps, st);
    QT_CASE(1, 8, true, false) QT_CASE(1, 2, true, false) QT_CASE(2, 8, true, false) QT_CASE(2, 4, true, false)
    QT_CASE(2, 2, true, false) QT_CASE(2, 1, true, false) QT_CASE(3, 4, true, false) QT_CASE(4, 4, true, false)
    QT_CASE(4, 1, true, false) QT_CASE(6, 2, true, false) QT_CASE(8, 2, true, false) QT_CASE(8, 1, true, false)
    QT_CASE(10, 2, true, false) QT_CASE(10, 1, true, false) QT_CASE(12, 1, true, false) QT_CASE(16, 1, true, false)
    QT_CASE(1, 4, false, false) QT_CASE(1, 1, false, false) QT_CASE(2, 4, false, false) QT_CASE(2, 1, false, false)
    QT_CASE(4, 2, false, false) QT_CASE(8, 1, false, false)
    QT_CASE(1, 4, true, true) QT_CASE(2, 4, true, true) QT_CASE(3, 4, true, true) QT_CASE(4, 4, true, true)
    QT_CASE(6, 2, true, true) QT_CASE(8, 2, true, true) QT_CASE(10, 2, true, true) QT_CASE(12, 1, true, true)
    QT_CASE(16, 1, true, true)
    QT_CASE(1, 2, false, true) QT_CASE(2, 2, false, true) QT_CASE(4, 1, false, true) QT_CASE(8, 1, false, true)
#undef QT_CASE
    return cudaErrorInvalidValue;
}

}  // namespace qt
