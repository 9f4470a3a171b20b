// qt_router_search.cu -- the search of the router form: the learned start cell
// and the Elkan certificate for the nearest-cell searches of Algorithm III
// (Pages & Wilbertz, arXiv:1101.3228, Sec. 3.2 searches by brute force; the
// paper's kd-tree attempt there is the prior art for a sub-linear search).
//
// One CTA of 128 threads (one warpgroup) per work item of 128 samples, thread t
// owning sample row t, several CTAs per SM:
//   1. draw the pair (X_k, X_{k+1}) of row t (qt_sampler.cuh);
//   2. the router MLP d -> 64 -> 64 -> 64 on the 5th-generation tensor cores,
//      both grids' rows at once: the whitened coordinates z = L^{-1}(x - mu)
//      and the hidden activations are FP16 rows of two 128-row operand tiles in
//      shared memory, the weights FP16 tiles (converted once per CTA), and each
//      layer is two tcgen05.mma chains (M = 128, N = 64, FP32 accumulators in
//      tensor memory: X's in columns 0-63, Y's in 64-127) issued by one thread;
//      every thread reads its row back with one tcgen05.ld, adds the bias and
//      applies the ReLU (the last layer: the two largest of the 64 logits);
//   3. per grid, the start cell i0 = the nearest member of the two predicted
//      buckets, then the walk over i0's neighbours in increasing distance up to
//      the triangle-inequality bound, and the FP32 margin certificate; an
//      exhausted list or an uncertified margin goes to the exact window search;
//   4. count p^k_ij.
// The network only proposes where to start: any bucket, any rounding of the
// FP16 inference, gives the exact cell (the certificate decides).
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "../../include/qt.h"
#include "qt_forward_tc.cuh"
#include "qt_launch.h"

namespace qt {

namespace {

constexpr int kRtK1 = 16;                  // operand columns of layer 1: z zero-padded (d <= 16)
constexpr int kRtRows = 128;               // samples per work item = MMA M
constexpr uint32_t kRtTmemCols = 128;      // accumulators: X rows in columns 0-63, Y rows in 64-127
// dynamic shared memory: FP16 weight tiles, FP32 biases, the two sample operand tiles
constexpr int kRtW1Bytes = kRtHidden * kRtK1 * 2;
constexpr int kRtW2Bytes = kRtHidden * kRtHidden * 2;
constexpr int kRtW3Bytes = kRtBuckets * kRtHidden * 2;
constexpr int kRtBiasBytes = (2 * kRtHidden + kRtBuckets) * 4;
constexpr int kRtTileBytes = kRtRows * kRtHidden * 2;
constexpr int kRtOffW2 = kRtW1Bytes;
constexpr int kRtOffW3 = kRtOffW2 + kRtW2Bytes;
constexpr int kRtOffBias = kRtOffW3 + kRtW3Bytes;
constexpr int kRtOffX = kRtOffBias + kRtBiasBytes;
constexpr int kRtOffY = kRtOffX + kRtTileBytes;
constexpr int kRtDynSmem = kRtOffY + kRtTileBytes;
static_assert(kRtOffW2 % 128 == 0 && kRtOffW3 % 128 == 0 && kRtOffBias % 128 == 0 && kRtOffX % 128 == 0 &&
                  kRtOffY % 128 == 0,
              "operand tiles on 128-byte boundaries");
static_assert(kRtHidden == 64 && kRtBuckets == 64, "one 64-column accumulator per grid");
// at most four CTAs share an SM's 512 tensor-memory columns: every CTA takes
// more than a fifth of the SM's shared memory
static_assert(5 * (kRtDynSmem + 1024) > 228 * 1024, "tensor-memory budget");

// Byte offset of element (r, c) of an FP16 operand with K columns in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// consecutive along K, then along the rows.
__device__ __forceinline__ uint32_t kmajor(int r, int c, int K)
{
    return (uint32_t)((((r >> 3) * (K >> 3) + (c >> 3)) << 7) + ((r & 7) << 4) + ((c & 7) << 1));
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b)
{
    return (uint32_t)__half_as_ushort(__float2half_rn(a)) | ((uint32_t)__half_as_ushort(__float2half_rn(b)) << 16);
}

// Row t of an operand tile with K columns from 8-column groups of values.
template <int K>
__device__ __forceinline__ void put_row(unsigned char* tile, int t, const float (&v)[K])
{
#pragma unroll
    for (int g = 0; g < K / 8; ++g)
        *reinterpret_cast<uint4*>(tile + kmajor(t, 8 * g, K)) =
            make_uint4(pack_h2(v[8 * g], v[8 * g + 1]), pack_h2(v[8 * g + 2], v[8 * g + 3]),
                       pack_h2(v[8 * g + 4], v[8 * g + 5]), pack_h2(v[8 * g + 6], v[8 * g + 7]));
}

// This thread's row of a 64-column accumulator (tensor-memory lane = row),
// loaded and waited for in one block so that nothing reads the registers early.
__device__ __forceinline__ void tmem_row64(uint32_t taddr, float (&v)[64])
{
    asm volatile(
        "{\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t}"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
          "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]),
          "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]),
          "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31]),
          "=f"(v[32]), "=f"(v[33]), "=f"(v[34]), "=f"(v[35]), "=f"(v[36]), "=f"(v[37]), "=f"(v[38]), "=f"(v[39]),
          "=f"(v[40]), "=f"(v[41]), "=f"(v[42]), "=f"(v[43]), "=f"(v[44]), "=f"(v[45]), "=f"(v[46]), "=f"(v[47]),
          "=f"(v[48]), "=f"(v[49]), "=f"(v[50]), "=f"(v[51]), "=f"(v[52]), "=f"(v[53]), "=f"(v[54]), "=f"(v[55]),
          "=f"(v[56]), "=f"(v[57]), "=f"(v[58]), "=f"(v[59]), "=f"(v[60]), "=f"(v[61]), "=f"(v[62]), "=f"(v[63])
        : "r"(taddr), "r"(taddr + 32u)
        : "memory");
}

// One layer of the MLP for both tiles: the rows every thread wrote are made
// visible to the tensor cores, thread 0 issues the two MMA chains (K columns,
// 16 per instruction) and commits them to `bar`; all threads wait for the
// accumulators.  The outcome of the bounded wait is the same for the whole CTA.
__device__ __forceinline__ bool mlp_layer(uint32_t tmem, uint32_t tileX, uint32_t tileY, uint32_t w, int K,
                                          uint32_t bar, uint32_t& phase, long long budget)
{
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        const uint32_t idesc = (1u << 4) | ((uint32_t)(kRtHidden >> 3) << 17) | ((uint32_t)(kRtRows >> 4) << 24);
        for (int s = 0; s < K / 16; ++s)
            tc_mma(tmem, smem_desc(tileX + s * 256, 128, K * 16), smem_desc(w + s * 256, 128, K * 16), idesc,
                   s > 0 ? 1u : 0u);
        for (int s = 0; s < K / 16; ++s)
            tc_mma(tmem + (uint32_t)kRtHidden, smem_desc(tileY + s * 256, 128, K * 16),
                   smem_desc(w + s * 256, 128, K * 16), idesc, s > 0 ? 1u : 0u);
        tc_commit(bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase, budget);
    phase ^= 1u;
    const bool all = __syncthreads_and(ok) != 0;
    tc_fence_after();
    return all;
}

// Bias + ReLU of this thread's accumulator row, written as the next layer's
// operand row (FP16, clamped inside the FP16 range).
__device__ __forceinline__ void hidden_row(uint32_t taddr, const float* __restrict__ bias, unsigned char* tile, int t)
{
    float v[64];
    tmem_row64(taddr, v);
#pragma unroll
    for (int o = 0; o < 64; ++o) v[o] = fminf(fmaxf(v[o] + bias[o], 0.0f), 60000.0f);
    put_row<64>(tile, t, v);
}

// The two largest logits of this thread's row (ties to the lower bucket).
__device__ __forceinline__ void top2_row(uint32_t taddr, const float* __restrict__ bias, int& bk, int& bk2)
{
    float v[64];
    tmem_row64(taddr, v);
    bk = 0;
    bk2 = 1;
    float mx = v[0] + bias[0], mx2 = v[1] + bias[1];
    if (mx2 > mx) {
        bk = 1;
        bk2 = 0;
        const float t = mx;
        mx = mx2;
        mx2 = t;
    }
#pragma unroll
    for (int o = 2; o < 64; ++o) {
        const float h = v[o] + bias[o];
        if (h > mx) {
            mx2 = mx;
            bk2 = bk;
            mx = h;
            bk = o;
        } else if (h > mx2) {
            mx2 = h;
            bk2 = o;
        }
    }
}

// Whitened, zero-padded layer-1 row of a sample for one grid: z = L^{-1}(x - mu) in FP32.
template <int DM>
__device__ __forceinline__ void whiten_row(const float (&v)[DM], const float* __restrict__ mu,
                                           const float* __restrict__ linv, int d, unsigned char* tile, int t)
{
    float xh[DM];
#pragma unroll
    for (int l = 0; l < DM; ++l) xh[l] = l < d ? __fsub_rn(v[l], mu[l]) : 0.0f;
    float z[kRtK1];
#pragma unroll
    for (int l = 0; l < kRtK1; ++l) {
        float a = 0.0f;
        if (l < DM) {
#pragma unroll
            for (int q = 0; q < DM; ++q)
                if (q <= l && l < d) a = fmaf(linv[l * d + q], xh[q], a);
        }
        z[l] = a;
    }
    put_row<kRtK1>(tile, t, z);
}

struct RouteOut {
    int cell;       // certified cell, or -1 (exact fallback needed)
    int cands;      // candidate distances evaluated
};

// Certified search of one point for grid G from the predicted buckets bk, bk2
// (records in global memory).  Start cell: the nearest member of the two
// buckets.  Walk: the neighbours of the start cell i0 in increasing distance
// while their distance to i0 is below r0 + r* (r0 >= |x - c_i0|, r* >= the best
// distance so far, both upper bounds from FP32 scores, slack 2^-20): every
// point beyond is farther from x than the best candidate.  Then the FP32 margin
// certificate on the best two candidate scores.
template <int DM>
__device__ __noinline__ RouteOut route_search(const ForwardParams& p, const GridInfo& G, int gidx,
                                              const float (&v)[DM], int bk, int bk2)
{
    RouteOut out;
    out.cell = -1;
    out.cands = 0;
    const int d = p.d;
    constexpr int F = Rec32<DM>::kFloats;
    const float* recs = p.rec32 + G.roff * F;
    float xs[DM];
    float A2 = 0.0f;
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        const float xh = l < d ? __fsub_rn(v[l], G.mu[l]) : 0.0f;
        xs[l] = -2.0f * xh;
        A2 = __fmaf_rn(xh, xh, A2);
    }
    const float A = __fsqrt_rn(A2);
    // a record is F floats on a 16-byte boundary: F / 4 vector loads
    auto score = [&](int j) {
        const float4* r4 = reinterpret_cast<const float4*>(recs + (long long)j * F);
        float f[F];
#pragma unroll
        for (int v = 0; v < F / 4; ++v) {
            const float4 a = __ldg(r4 + v);
            f[4 * v] = a.x;
            f[4 * v + 1] = a.y;
            f[4 * v + 2] = a.z;
            f[4 * v + 3] = a.w;
        }
        float sc = f[0];
#pragma unroll
        for (int l = 0; l < DM; ++l) sc = __fmaf_rn(xs[l], f[1 + l], sc);
        return sc;
    };
    // start cell: nearest member of the two most likely buckets
    int i0 = -1;
    float s0 = __int_as_float(0x7F800000);
    for (int pass = 0; pass < 2; ++pass) {
        const int b = pass == 0 ? bk : bk2;
        const int bs = p.rt_bstart[b], be = p.rt_bstart[b + 1];
        for (int t = bs; t < be; ++t) {
            const int j = p.rt_members[t];
            const float sc = score(j);
            if (sc < s0) {
                s0 = sc;
                i0 = j;
            }
        }
        out.cands += be - bs;
    }
    if (i0 < 0) return out;
    // Elkan walk over the neighbours of i0
    const float Eg = (float)(d + 2) * 0x1p-22f * (A + G.R) * (A + G.R);
    auto rub = [&](float sc) { return __fsqrt_rn(fmaxf(sc + A2 + Eg, 0.0f)) * (1.0f + 0x1p-20f); };
    const float r0 = rub(s0);
    float B1 = s0, S = __int_as_float(0x7F800000), rs = r0;
    int i1 = i0;
    const long long base = ((long long)gidx * p.rt_N + i0) * p.rt_C;
    // neighbours in blocks of 8 independent loads, then tested in order
    constexpr int kW = 8;
    const bool vec8 = (p.rt_C & 7) == 0;     // every list starts on a 32-byte boundary
    int scanned = 0;                 // neighbours taken as candidates
    bool stop = false;               // the distance bound was reached inside the list
    const int lim = p.rt_C;
    for (int c = 0; c < lim && !stop; c += kW) {
        float dl[kW], sc[kW];
        int jj[kW];
        if (vec8 && c + kW <= lim) {
            // whole blocks of 8 on 16-byte boundaries: two vector loads per list
            const float4* d4 = reinterpret_cast<const float4*>(p.rt_nb_dist + base + c);
            const int4* j4 = reinterpret_cast<const int4*>(p.rt_nb_idx + base + c);
            const float4 da = __ldg(d4), db = __ldg(d4 + 1);
            const int4 ja = __ldg(j4), jb = __ldg(j4 + 1);
            dl[0] = da.x; dl[1] = da.y; dl[2] = da.z; dl[3] = da.w;
            dl[4] = db.x; dl[5] = db.y; dl[6] = db.z; dl[7] = db.w;
            jj[0] = ja.x; jj[1] = ja.y; jj[2] = ja.z; jj[3] = ja.w;
            jj[4] = jb.x; jj[5] = jb.y; jj[6] = jb.z; jj[7] = jb.w;
        } else {
#pragma unroll
            for (int q = 0; q < kW; ++q) {
                const int cq = min(c + q, lim - 1);
                dl[q] = __ldg(p.rt_nb_dist + base + cq);
                jj[q] = __ldg(p.rt_nb_idx + base + cq);
            }
        }
#pragma unroll
        for (int q = 0; q < kW; ++q) sc[q] = score(jj[q]);
#pragma unroll
        for (int q = 0; q < kW; ++q) {
            if (stop || c + q >= lim) continue;
            if (dl[q] > (r0 + rs) * (1.0f + 0x1p-20f)) {
                stop = true;
                continue;
            }
            ++scanned;
            if (sc[q] < B1) {
                S = B1;
                B1 = sc[q];
                i1 = jj[q];
                rs = rub(B1);
            } else {
                S = fminf(S, sc[q]);
            }
        }
    }
    out.cands += scanned;
    if (!stop) return out;          // list exhausted before the bound: exact fallback
    const float* r = recs + (long long)i1 * F;
    float n2 = 0.0f;
#pragma unroll
    for (int l = 0; l < DM; ++l) n2 = __fmaf_rn(r[1 + l], r[1 + l], n2);
    if (screen_certified(d, A, B1, S, __fsqrt_rn(n2))) out.cell = i1;
    return out;
}

template <int DM>
__global__ void __launch_bounds__(kRtRows, 4) forward_router_kernel(const ForwardParams p)
{
    extern __shared__ __align__(1024) unsigned char dsm_rt[];
    __shared__ __align__(16) float s_linvA[DM * DM], s_linvB[DM * DM];
    __shared__ long long s_item;
    __shared__ LayerDesc s_L;
    __shared__ GridInfo s_GA, s_GB;
    __shared__ __align__(16) float s_pf[param_count(DM)];
    __shared__ __align__(8) unsigned long long s_mma;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int d = p.d;
    // the grids must be those the router was built for (checked before any
    // tensor memory is taken)
    if (p.status->spare[0] != p.rt_checksum) {
        if (tid == 0) record_error(p.status, 1 /* QT_EINVAL */, 21);
        return;
    }
    unsigned char* sW1 = dsm_rt;
    unsigned char* sW2 = dsm_rt + kRtOffW2;
    unsigned char* sW3 = dsm_rt + kRtOffW3;
    float* sBias = reinterpret_cast<float*>(dsm_rt + kRtOffBias);   // b1 [64], b2 [64], b3 [64]
    unsigned char* sX = dsm_rt + kRtOffX;
    unsigned char* sY = dsm_rt + kRtOffY;
    // FP16 weight tiles (row = output unit, column = input unit), FP32 biases
    {
        const float* W1 = p.rt_params;
        const float* b1 = W1 + kRtHidden * d;
        const float* W2 = b1 + kRtHidden;
        const float* b2 = W2 + kRtHidden * kRtHidden;
        const float* W3 = b2 + kRtHidden;
        const float* b3 = W3 + kRtBuckets * kRtHidden;
        for (int e = tid; e < kRtHidden * kRtK1; e += kRtRows) {
            const int o = e / kRtK1, l = e % kRtK1;
            *reinterpret_cast<__half*>(sW1 + kmajor(o, l, kRtK1)) = __float2half_rn(l < d ? W1[o * d + l] : 0.0f);
        }
        for (int e = tid; e < kRtHidden * kRtHidden; e += kRtRows) {
            const int o = e / kRtHidden, i = e % kRtHidden;
            *reinterpret_cast<__half*>(sW2 + kmajor(o, i, kRtHidden)) = __float2half_rn(W2[e]);
            *reinterpret_cast<__half*>(sW3 + kmajor(o, i, kRtHidden)) = __float2half_rn(W3[e]);
        }
        for (int e = tid; e < kRtHidden; e += kRtRows) {
            sBias[e] = b1[e];
            sBias[kRtHidden + e] = b2[e];
            sBias[2 * kRtHidden + e] = b3[e];
        }
    }
    if (tid == 0) {
        mbar_init(smem_u32(&s_mma), 1);
        fence_proxy_async();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kRtTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);     // this warp's lanes
    const uint32_t uW1 = smem_u32(sW1), uW2 = smem_u32(sW2), uW3 = smem_u32(sW3);
    const uint32_t uX = smem_u32(sX), uY = smem_u32(sY);
    const uint32_t bar = smem_u32(&s_mma);
    uint32_t phase = 0;
    bool mma_lost = false;          // a wait gave up with MMAs possibly in flight
    int cur = -1;
    while (true) {
        if (tid == 0) {
            long long it = -1;
            if (*((volatile int32_t*)&p.status->code) == 0) it = (long long)atomicAdd(&p.status->queue, 1ull);
            s_item = it;
        }
        __syncthreads();
        const long long item = s_item;
        if (item < 0 || item >= p.total_items) break;
        int k = (cur >= 0 && item >= s_L.item_begin && item < s_L.item_begin + s_L.items) ? cur : -1;
        if (k < 0) {
            int lo = 0, hi = p.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.layers[mid].item_begin <= item) lo = mid; else hi = mid - 1;
            }
            k = lo;
        }
        if (k != cur) {
            __syncthreads();
            if (tid == 0) {
                s_L = p.layers[k];
                s_GA = p.grids[s_L.gridA];
                s_GB = p.grids[s_L.gridB];
            }
            const int pc = param_count(d);
            for (int e = tid; e < pc; e += kRtRows) s_pf[e] = p.params_f[(long long)k * p.params_stride + e];
            for (int e = tid; e < d * d; e += kRtRows) {
                s_linvA[e] = p.rt_linv[(long long)k * d * d + e];
                s_linvB[e] = p.rt_linv[(long long)(k + 1) * d * d + e];
            }
            __syncthreads();
            cur = k;
        }
        const LayerDesc& L = s_L;
        const unsigned long long ms = (unsigned long long)(item - L.item_begin) * kRtRows + tid;
        const bool valid = ms < p.M;
        float X[DM], Y[DM];
        pair_f32<DM>(s_pf, d, p.seed, k, valid ? ms : 0ull, X, Y);
        // ---- router MLP on the tensor cores, both grids' rows together
        whiten_row<DM>(X, s_GA.mu, s_linvA, d, sX, tid);
        whiten_row<DM>(Y, s_GB.mu, s_linvB, d, sY, tid);
        if (!mlp_layer(tmem, uX, uY, uW1, kRtK1, bar, phase, p.spin_budget)) {
            mma_lost = true;
            break;
        }
        hidden_row(trow, sBias, sX, tid);
        hidden_row(trow + kRtHidden, sBias, sY, tid);
        if (!mlp_layer(tmem, uX, uY, uW2, kRtHidden, bar, phase, p.spin_budget)) {
            mma_lost = true;
            break;
        }
        hidden_row(trow, sBias + kRtHidden, sX, tid);
        hidden_row(trow + kRtHidden, sBias + kRtHidden, sY, tid);
        if (!mlp_layer(tmem, uX, uY, uW3, kRtHidden, bar, phase, p.spin_budget)) {
            mma_lost = true;
            break;
        }
        int bkA, bk2A, bkB, bk2B;
        top2_row(trow, sBias + 2 * kRtHidden, bkA, bk2A);
        top2_row(trow + kRtHidden, sBias + 2 * kRtHidden, bkB, bk2B);
        tc_fence_before();          // the next item's MMAs overwrite these accumulators
        // ---- certified searches
        int ci = 0, cj = 0, cand = 0;
        bool needA = false, needB = false;
        if (L.NA > 1) {
            const RouteOut r = route_search<DM>(p, s_GA, L.gridA, X, bkA, bk2A);
            ci = r.cell;
            cand += r.cands;
            needA = r.cell < 0 && valid;
        }
        if (L.NB > 1) {
            const RouteOut r = route_search<DM>(p, s_GB, L.gridB, Y, bkB, bk2B);
            cj = r.cell;
            cand += r.cands;
            needB = r.cell < 0 && valid;
        }
        // candidates per search (statistics)
        int wc = valid ? cand : 0;
        for (int off = 16; off >= 1; off >>= 1) wc += __shfl_xor_sync(0xFFFFFFFFu, wc, off);
        if (lane == 0) atomicAdd(&p.status->candidates, (unsigned long long)wc);
        // exact window search for the uncertified
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const bool need = g == 0 ? needA : needB;
            unsigned mask = __ballot_sync(0xFFFFFFFFu, need);
            if (!mask) continue;
            double z[DM];
#pragma unroll
            for (int l = 0; l < DM; ++l) z[l] = (double)(g == 0 ? X[l] : Y[l]);
            const GridInfo& G = g == 0 ? s_GA : s_GB;
            float xs[DM];
            float A2 = 0.0f;
#pragma unroll
            for (int l = 0; l < DM; ++l) {
                const float xh = l < d ? __fsub_rn(g == 0 ? X[l] : Y[l], G.mu[l]) : 0.0f;
                xs[l] = -2.0f * xh;
                A2 = __fmaf_rn(xh, xh, A2);
            }
            const float A = __fsqrt_rn(A2);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const int r = warp_window_nn<DM>(xs, A, z, src, p.rec32 + G.roff * Rec32<DM>::kFloats, G.Npad,
                                                 p.g64 + G.goff * d, G.N, d);
                if (lane == src) {
                    if (g == 0) ci = r; else cj = r;
                }
                if (lane == 0) atomicAdd(&p.status->rechecks, 1ull);
            }
        }
        if (valid) {
            if ((unsigned)ci >= (unsigned)L.NA || (unsigned)cj >= (unsigned)L.NB) {
                record_error(p.status, 6 /* QT_EDEVICE */, 22);
            } else {
                count_add(p.counts, p.counts_u32, L.coff + (long long)ci * L.NB + cj, 1u);
                if (p.dump_count > 0 && (ms % (unsigned long long)p.dump_stride) == 0ull) {
                    const unsigned long long t = ms / (unsigned long long)p.dump_stride;
                    if (t < (unsigned long long)p.dump_count) {
                        const long long row = (long long)k * p.dump_count + (long long)t;
                        for (int l = 0; l < d; ++l) {
                            p.dumpX[row * d + l] = (double)X[l];
                            p.dumpY[row * d + l] = (double)Y[l];
                        }
                        p.dumpI[row] = ci;
                        p.dumpJ[row] = cj;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (mma_lost) {
        // a wait gave up: record it, and let the committed MMAs finish before the
        // tensor memory is released (the parity of the phase that gave up)
        if (tid == 0) record_error(p.status, 4 /* QT_ETIMEOUT */, 23);
        mbar_wait_bounded(bar, phase ^ 1u, kDrainUs);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kRtTmemCols)
                     : "memory");
    }
}

template <int DM>
cudaError_t launch_rt(const ForwardParams& p, int num_sms, int* bps, cudaStream_t st)
{
    auto kern = forward_router_kernel<DM>;
    const int dyn = kRtDynSmem;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    // CTAs per SM from the kernel's registers and shared memory (the runtime's
    // occupancy query answers 1 for this kernel, although four fit), at most
    // as many as share the SM's 512 tensor-memory columns
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, regs_sm = 0, smem_sm = 0, smem_rsv = 0, thr_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
        return e;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;          // registers are granted per warp
    int b = 512 / (int)kRtTmemCols;
    b = std::min(b, regs_sm / (warp_regs * (kRtRows / 32)));
    b = std::min(b, smem_sm / (int)(dyn + fa.sharedSizeBytes + smem_rsv));
    b = std::min(b, thr_sm / kRtRows);
    if (b < 1) return cudaErrorInvalidConfiguration;
    *bps = b;
    long long grid = (long long)num_sms * b;
    if (grid > p.total_items) grid = p.total_items;
    kern<<<(unsigned)grid, kRtRows, dyn, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_router_forward(int dm, const ForwardParams& p, int num_sms, int* bps, cudaStream_t st)
{
    if (dm == 2) return launch_rt<2>(p, num_sms, bps, st);
    if (dm == 4) return launch_rt<4>(p, num_sms, bps, st);
    if (dm == 6) return launch_rt<6>(p, num_sms, bps, st);
    if (dm == 8) return launch_rt<8>(p, num_sms, bps, st);
    if (dm == 10) return launch_rt<10>(p, num_sms, bps, st);
    if (dm == 12) return launch_rt<12>(p, num_sms, bps, st);
    if (dm == 16) return launch_rt<16>(p, num_sms, bps, st);
    return cudaErrorInvalidValue;
}

}  // namespace qt
