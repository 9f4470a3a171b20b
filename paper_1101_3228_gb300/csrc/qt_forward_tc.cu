// qt_forward_tc.cu -- the forward step of Algorithm III (Pages & Wilbertz,
// arXiv:1101.3228, Sec. 4) with the nearest-cell screen on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// The screen scores s_j = |g_j|^2 - 2 x^.g_j (g_j, x^ centred on the grid's
// FP32 centre) are one GEMM per 128 samples x 256 grid points: sample rows
// [a_hi, a_hi, a_lo, 1, 1] times grid rows [g_hi, g_lo, g_hi, cc_hi, cc_lo],
// a = -2 sigma x^, g = sigma g^, cc = sigma^2 |g^|^2, each split into an FP16
// head and an FP16 tail, sigma = 2^tc_exp so that the grid fits in [-1, 1].
// The three cross products reproduce the FP32 score to about 2^-21 relative
// (the tail x tail product is below 2^-22); K = 16 holds 3d + 2 columns for
// d <= 4, K = 32 for d <= 10.
//
// Per work item (layer k, 128 samples): one thread per sample draws the pair,
// writes both sample rows into shared memory, and the CTA walks the operand
// tiles of Gamma_k and Gamma_{k+1}: thread 0 issues the MMA of tile t + 1 into
// one of two 256-column TMEM accumulators while all 128 threads read tile t
// with tcgen05.ld and keep, per sample, the running minimum per 16-column chunk
// (best, smallest other chunk minimum, best chunk).  Operand tiles arrive by
// bulk copies (TMA engine); they stay in shared memory for the whole layer when
// both grids fit, else they stream through a ring.
//
// Exactness: the best chunk is re-scored on the CUDA cores in FP32 (index and
// second score inside the chunk), and the pick is certified against the exact
// FP64 distance with the FP32 bound inside the chunk and the tensor-core bound
// outside it; uncertified samples get a warp-wide FP32 re-screen of the whole
// grid and, if that cannot certify either, the exact FP64 search.
#include <cuda_fp16.h>

#include "qt_forward.cuh"
#include "qt_launch.h"

namespace qt {

namespace {

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    // tcgen05 shared-memory matrix descriptor, canonical K-major layout, no swizzle
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float min16(const float* v)
{
    const float a = min3f(v[0], v[1], v[2]);
    const float b = min3f(v[3], v[4], v[5]);
    const float c = min3f(v[6], v[7], v[8]);
    const float e = min3f(v[9], v[10], v[11]);
    const float f = min3f(v[12], v[13], v[14]);
    return min3f(min3f(a, b, c), min3f(e, f, v[15]), __int_as_float(0x7F800000));
}

// Bound on |tensor-core score - exact score| in FP32-score units for a grid
// point at distance r from the centre (A = |x^|): the FP32 bound (d+2) 2^-24
// plus 32 FP32 additions of the MMA (2^-23 each, counted as truncations), the
// dropped tail product and the head/tail representation (3 * 2^-22), and the
// absolute floor of the FP16 tails (2^-25 each) divided by sigma^2.
__device__ __forceinline__ float tc_bound(int d, float A, float r, float inv_sigma)
{
    const float rel = 1.5f * 0x1p-18f;
    const float absf = (0x1p-23f * sqrtf((float)d) * (A + r) * (1.0f / inv_sigma) + 0x1p-24f) * inv_sigma * inv_sigma;
    return rel * (r * r + 2.0f * A * r) + absf;
}

__device__ __forceinline__ float cc_bound(int d, float A, float r)
{
    return (float)(d + 2) * 0x1p-24f * (1.0f + 0x1p-10f) * (r * r + 2.0f * A * r);
}

// FP32 scores of one 16-record chunk of a grid (records in global memory):
// lowest-index minimum, the smallest other score, the norm of the best record.
template <int DM>
__device__ __forceinline__ void cc_chunk(const float* __restrict__ recs, int chunk, const float (&x)[DM], int& idx,
                                         float& best, float& S1, float& r1)
{
    constexpr int F = Rec32<DM>::kFloats;
    idx = -1;
    best = __int_as_float(0x7F800000);
    S1 = __int_as_float(0x7F800000);
    int bq = 0;
    for (int q = 0; q < kChunk; ++q) {
        const float* r = recs + (chunk * kChunk + q) * F;
        float sc = r[0];
#pragma unroll
        for (int l = 0; l < DM; ++l) sc = __fmaf_rn(x[l], r[1 + l], sc);
        if (sc < best) {
            S1 = fminf(S1, best);
            best = sc;
            bq = q;
        } else {
            S1 = fminf(S1, sc);
        }
    }
    idx = chunk * kChunk + bq;
    const float* r = recs + idx * F;
    float n2 = 0.0f;
#pragma unroll
    for (int l = 0; l < DM; ++l) n2 = __fmaf_rn(r[1 + l], r[1 + l], n2);
    r1 = __fsqrt_rn(n2);
}

// Mixed certificate: FP32 scores inside the two best chunks (best, S1: the
// smallest other FP32 score there), tensor-core scores outside them (B2tc: the
// smallest chunk minimum of the other chunks, FP32-score units).
__device__ __forceinline__ bool tc_certified(int d, float A, float best, float S1, float B2tc, float r1,
                                             float inv_sigma, int& why)
{
    const float Ap = A * (1.0f + 0x1p-18f);
    const float r1p = r1 * (1.0f + 0x1p-18f);
    const float E1 = cc_bound(d, Ap, r1p);
    const float U = best + E1;
    const float A2 = Ap * Ap;
    const float eta = 0x1p-44f * (A2 + fabsf(best) + E1);
    const float rad = fmaxf(A2 + U + 0x1p-18f * (A2 + fabsf(U)) + eta, 0.0f);
    const float rho = Ap + __fsqrt_rn(rad);
    const float lo_in = S1 - cc_bound(d, Ap, rho);
    const float lo_out = B2tc - tc_bound(d, Ap, rho, inv_sigma);
    const float rhs = U + eta;
    // additive slack for the FP32 evaluation of both sides
    const bool ok_in = lo_in - rhs > 0x1p-20f * (fabsf(lo_in) + fabsf(rhs)) + eta || lo_in == __int_as_float(0x7F800000);
    const bool ok_out = lo_out - rhs > 0x1p-20f * (fabsf(lo_out) + fabsf(rhs)) + eta || lo_out == __int_as_float(0x7F800000);
    why = ok_in ? (ok_out ? 0 : 2) : 1;
    return ok_in && ok_out;
}

}  // namespace

// FP16 operand tiles of every grid: row j of grid g (tile j/256) holds
// [g_hi (d), g_lo (d), g_hi (d), cc_hi, cc_lo, 0 ...] of sigma g^ and
// sigma^2 cc; padded rows carry cc_hi = +inf.  Layout inside a tile: core
// matrices of 8 rows x 8 halves, (row block, K block) at ((n/8)(K/8) + k/8) * 64.
__global__ void prep_tc_tiles_kernel(const float* __restrict__ rec32, GridInfo* gi, int ngrids, int d,
                                     int rec_floats, int K, long long total_rows, __half* tiles)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total_rows) return;
    int lo = 0, hi = ngrids - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gi[mid].tc_toff * kTcTileN <= r) lo = mid; else hi = mid - 1;
    }
    const GridInfo& G = gi[lo];
    const long long j = r - G.tc_toff * kTcTileN;
    // sigma = 2^e with sigma R <= 1
    int e = 0;
    if (G.R > 0.0f) {
        int ex;
        frexpf(G.R, &ex);   // R = f 2^ex, f in [0.5, 1)
        e = -ex;
    }
    if (j == 0) gi[lo].tc_exp = e;
    const float sg = ldexpf(1.0f, e);
    const long long tile = G.tc_toff + j / kTcTileN;
    const int n = (int)(j % kTcTileN);
    __half* t = tiles + tile * (long long)kTcTileN * K;
    auto put = [&](int k, __half v) { t[((n >> 3) * (K >> 3) + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7)] = v; };
    for (int k = 0; k < K; ++k) put(k, __float2half_rn(0.0f));
    if (j < G.N) {
        const float* rc = rec32 + (G.roff + j) * rec_floats;
        for (int l = 0; l < d; ++l) {
            const float v = sg * rc[1 + l];
            const __half h = __float2half_rn(v);
            const __half lo16 = __float2half_rn(v - __half2float(h));
            put(l, h);
            put(d + l, lo16);
            put(2 * d + l, h);
        }
        const float c = sg * sg * rc[0];
        const __half ch = __float2half_rn(c);
        put(3 * d, ch);
        put(3 * d + 1, __float2half_rn(c - __half2float(ch)));
    } else {
        put(3 * d, __float2half_rn(__int_as_float(0x7F800000)));
    }
}

template <int DM, int KT>
__global__ void __launch_bounds__(256, 1) forward_tc_kernel(const ForwardParams p)
{
    constexpr int K = 16 * KT;
    constexpr int kTileBytes = kTcTileN * K * 2;
    constexpr int kAbytes = kTcTileM * K * 2;
    extern __shared__ __align__(128) unsigned char dsm_tc[];
    __shared__ __align__(8) unsigned long long s_bfull[16];
    __shared__ __align__(8) unsigned long long s_mma[2];
    __shared__ uint32_t s_tmem;
    __shared__ long long s_item;
    __shared__ LayerDesc s_L;
    __shared__ GridInfo s_GA, s_GB;
    __shared__ __align__(16) float s_pf[param_count(DM)];
    __shared__ __align__(16) double s_pd[param_count(DM)];
    __shared__ int s_abort;
    __shared__ float s_mB1[kTcTileM], s_mBs[kTcTileM], s_mB3[kTcTileM];   // half-tile hand-over
    __shared__ int s_mbc[kTcTileM], s_mbcs[kTcTileM];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int d = p.d;
    const int RS = p.tc_slots;
    unsigned char* sA = dsm_tc;                     // two sample operands (grid A, grid B)
    unsigned char* sB = dsm_tc + 2 * kAbytes;         // operand tile ring
    const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);

    if (tid == 0) {
        for (int t = 0; t < RS; ++t) mbar_init(smem_u32(&s_bfull[t]), 1);
        mbar_init(smem_u32(&s_mma[0]), 1);
        mbar_init(smem_u32(&s_mma[1]), 1);
        fence_proxy_async();
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((uint32_t)(2 * kTcTileN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    uint32_t bphase = 0;                   // bit t: parity of slot t's barrier
    uint32_t mphase = 0;                   // bit b: parity of accumulator b's barrier
    uint32_t idesc = (1u << 4) | ((uint32_t)(kTcTileN >> 3) << 17) | ((uint32_t)(kTcTileM >> 4) << 24);
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
        const bool new_layer = k != cur;
        if (new_layer) {
            __syncthreads();
            if (tid == 0) {
                s_L = p.layers[k];
                s_GA = p.grids[s_L.gridA];
                s_GB = p.grids[s_L.gridB];
            }
            if (p.source == kSampler) {
                const int pc = param_count(d);
                for (int e = tid; e < pc; e += blockDim.x) {
                    s_pf[e] = p.params_f[(long long)k * p.params_stride + e];
                    s_pd[e] = p.params_d[(long long)k * p.params_stride + e];
                }
            }
            __syncthreads();
            cur = k;
        }
        const LayerDesc& L = s_L;
        const int tA = s_GA.tc_tiles, tB = s_GB.tc_tiles, nT = tA + tB;
        const bool resident = p.tc_resident != 0;
        auto tile_src = [&](int i) -> const unsigned char* {
            const long long gt = i < tA ? s_GA.tc_toff + i : s_GB.tc_toff + (i - tA);
            return reinterpret_cast<const unsigned char*>(p.tc_tiles) + gt * (long long)kTileBytes;
        };
        // ---- operand tiles: all of them once per layer (resident) or the first RS (streamed)
        if (tid == 0 && (!resident || new_layer)) {
            fence_proxy_async();
            const int first = resident ? nT : min(RS, nT);
            for (int i = 0; i < first; ++i) {
                const uint32_t b = smem_u32(&s_bfull[i]);
                mbar_arrive_expect_tx(b, kTileBytes);
                bulk_g2s(sB_u + i * kTileBytes, tile_src(i), kTileBytes, b);
            }
        }
        bool loaded_now = !resident || new_layer;    // barriers of this item's tiles still to be waited

        // ---- two warpgroups per sample row t: warpgroup 0 owns grid A (writes its
        // operand row, reads accumulator columns 0-127, resolves and rechecks the
        // A search), warpgroup 1 owns grid B (columns 128-255); both draw sample t
        const int wg = tid >> 7;
        const int t = tid & 127;
        const unsigned long long mtile = (unsigned long long)(item - L.item_begin) * kTcTileM;
        const unsigned long long ms = mtile + (unsigned long long)t;
        const bool valid = ms < p.M;
        const Centred<DM> cs = centred_sample_inl<DM>(p, s_pf, s_pd, s_GA.mu, s_GB.mu, k, valid ? ms : mtile);
        float xown[DM];   // -2 (sample - mu) for this warpgroup's grid
#pragma unroll
        for (int l = 0; l < DM; ++l) xown[l] = wg == 0 ? cs.xa[l] : cs.yb[l];
        const float Aown = wg == 0 ? cs.Aa : cs.Ab;
        const GridInfo& Gown = wg == 0 ? s_GA : s_GB;
        bool big = false;     // outside the FP16 range: skip the screen, search exactly
        {
            const float sg = ldexpf(1.0f, Gown.tc_exp);
            unsigned char* base = sA + wg * kAbytes;
#pragma unroll
            for (int kb = 0; kb < K / 8; ++kb)
                *reinterpret_cast<uint4*>(base + (((t >> 3) * (K / 8) + kb) * 64 + (t & 7) * 8) * 2) =
                    make_uint4(0u, 0u, 0u, 0u);
            __half* hrow = reinterpret_cast<__half*>(base);
            auto at = [&](int q) -> __half& { return hrow[((t >> 3) * (K / 8) + (q >> 3)) * 64 + (t & 7) * 8 + (q & 7)]; };
#pragma unroll
            for (int l = 0; l < DM; ++l) big = big || !(fabsf(sg * xown[l]) <= 16384.0f);
#pragma unroll
            for (int l = 0; l < DM; ++l) {
                if (l < d) {
                    const float v = big ? 0.0f : sg * xown[l];
                    const __half h = __float2half_rn(v);
                    at(l) = h;
                    at(d + l) = h;
                    at(2 * d + l) = __float2half_rn(v - __half2float(h));
                }
            }
            at(3 * d) = __float2half_rn(1.0f);
            at(3 * d + 1) = __float2half_rn(1.0f);
        }
        fence_proxy_async();     // generic-proxy writes of the operand rows -> tensor core
        __syncthreads();

        // ---- walk the tiles: MMA of tile i+1 overlaps the epilogue of tile i
        // per sample and half tile: best chunk (B1, bc), second chunk (Bs, bcs),
        // smallest other chunk minimum B3
        float B1 = __int_as_float(0x7F800000), Bs = __int_as_float(0x7F800000), B3 = __int_as_float(0x7F800000);
        int bc = 0, bcs = 1;
        int cown = -1;             // this warpgroup's cell for sample t
        bool need = false;
        auto issue = [&](int i) {
            // thread 0 only: wait for the tile, then the MMA into accumulator i & 1
            const int slot = resident ? i : i % RS;
            if (loaded_now || !resident) {
                const uint32_t b = smem_u32(&s_bfull[slot]);
                if (!mbar_wait_bounded(b, (bphase >> slot) & 1u, p.spin_budget)) {
                    record_error(p.status, 4 /* QT_ETIMEOUT */, 11);
                    s_abort = 1;
                    mbar_wait_bounded(b, (bphase >> slot) & 1u, 1ll << 24);
                }
            }
            tc_fence_after();
            const uint32_t a_base = sA_u + (i < tA ? 0 : kAbytes);
            const uint32_t b_base = sB_u + slot * kTileBytes;
            const uint32_t dt = tmem + (uint32_t)((i & 1) * kTcTileN);
#pragma unroll
            for (int s = 0; s < KT; ++s) {
                const uint64_t ad = smem_desc(a_base + s * 256, 128, K * 16);
                const uint64_t bd = smem_desc(b_base + s * 256, 128, K * 16);
                tc_mma(dt, ad, bd, idesc, s > 0 ? 1u : 0u);
            }
            tc_commit(smem_u32(&s_mma[i & 1]));
        };
        if (tid == 0) issue(0);
        for (int i = 0; i < nT; ++i) {
            const int slot = resident ? i : i % RS;
            if (tid == 0 && i + 1 < nT) issue(i + 1);
            // the barrier parities of tile i's slot advance once per load
            if (loaded_now || !resident) bphase ^= (1u << slot);
            const bool ok = mbar_wait_bounded(smem_u32(&s_mma[i & 1]), (mphase >> (i & 1)) & 1u, p.spin_budget);
            if (!ok) {
                if (tid == 0) {
                    record_error(p.status, 4 /* QT_ETIMEOUT */, 12);
                    s_abort = 1;
                }
                mbar_wait_bounded(smem_u32(&s_mma[i & 1]), (mphase >> (i & 1)) & 1u, 1ll << 24);
            }
            mphase ^= (1u << (i & 1));
            tc_fence_after();
            // epilogue: this thread's row, its warpgroup's 128 columns, 8 chunks
            const int lt = i < tA ? i : i - tA;
#pragma unroll
            for (int q = 0; q < kTcTileN / 64; q += 2) {
                float va[32], vb[32];
                tc_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                            (uint32_t)((i & 1) * kTcTileN + wg * (kTcTileN / 2) + q * 32),
                        va);
                tc_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                            (uint32_t)((i & 1) * kTcTileN + wg * (kTcTileN / 2) + (q + 1) * 32),
                        vb);
                tc_wait_ld();
                const float mcs[4] = {min16(va), min16(va + 16), min16(vb), min16(vb + 16)};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float mc = mcs[h];
                    const int c = lt * (kTcTileN / kChunk) + wg * (kTcTileN / 2 / kChunk) + q * 2 + h;
                    const bool t1 = mc < B1, t2 = mc < Bs;
                    B3 = fminf(B3, fmaxf(mc, Bs));
                    Bs = fminf(Bs, fmaxf(mc, B1));
                    bcs = t1 ? bc : (t2 ? c : bcs);
                    B1 = fminf(B1, mc);
                    bc = t1 ? c : bc;
                }
            }
            const bool endA = i == tA - 1, endB = i == nT - 1;
            // the partner warpgroup hands its half-tile state to the owner of this grid
            if ((endA && wg == 1) || (endB && wg == 0)) {
                s_mB1[t] = B1;
                s_mBs[t] = Bs;
                s_mB3[t] = B3;
                s_mbc[t] = bc;
                s_mbcs[t] = bcs;
            }
            tc_fence_before();
            __syncthreads();      // accumulator i & 1, (streamed) slot of tile i and the hand-over are ready
            if (tid == 0 && !resident && i + RS < nT) {
                const uint32_t b = smem_u32(&s_bfull[slot]);
                fence_proxy_async();
                mbar_arrive_expect_tx(b, kTileBytes);
                bulk_g2s(sB_u + slot * kTileBytes, tile_src(i + RS), kTileBytes, b);
            }
            if ((endA && wg == 0) || (endB && wg == 1)) {
                // merge the two half-tile states: the two smallest chunk minima
                // (ties to the lower chunk), the rest into B3
                float v4[4] = {B1, Bs, s_mB1[t], s_mBs[t]};
                int c4[4] = {bc, bcs, s_mbc[t], s_mbcs[t]};
                float rest = fminf(B3, s_mB3[t]);
                int f = 0;
#pragma unroll
                for (int q = 1; q < 4; ++q)
                    if (v4[q] < v4[f] || (v4[q] == v4[f] && c4[q] < c4[f])) f = q;
                int g2 = f == 0 ? 1 : 0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q != f && (v4[q] < v4[g2] || (v4[q] == v4[g2] && c4[q] < c4[g2]))) g2 = q;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q != f && q != g2) rest = fminf(rest, v4[q]);
                const int mbc = c4[f], mbcs = c4[g2];
                // re-score the two best chunks in FP32 and certify
                const float inv_sg = ldexpf(1.0f, -Gown.tc_exp);
                const float* recs = p.rec32 + Gown.roff * Rec32<DM>::kFloats;
                const int nch = Gown.Npad / kChunk;      // chunks with FP32 records
                int idx, idx2;
                float best, S1, r1, best2, S12, r12;
                cc_chunk<DM>(recs, mbc, xown, idx, best, S1, r1);
                if (mbcs < nch && mbcs != mbc) {
                    cc_chunk<DM>(recs, mbcs, xown, idx2, best2, S12, r12);
                } else {
                    idx2 = idx;
                    best2 = S12 = __int_as_float(0x7F800000);
                    r12 = r1;
                }
                float in2;
                if (best2 < best || (best2 == best && idx2 < idx)) {
                    in2 = fminf(S12, best);
                    best = best2;
                    idx = idx2;
                    r1 = r12;
                } else {
                    in2 = fminf(S1, best2);
                }
                const float B3cc = rest * inv_sg * inv_sg;
                int why = 0;
                const bool tcok = tc_certified(d, Aown, best, in2, B3cc, r1, inv_sg, why);
                const bool rng_ok = idx < Gown.N && !big;
                const bool cert = tcok && rng_ok;
                if (valid && !cert) atomicAdd(&p.status->spare[!rng_ok ? 3 : why], 1ull);
                cown = idx;
                need = !cert && valid;
            }
            if (endA || endB) {
                B1 = Bs = B3 = __int_as_float(0x7F800000);
                bc = 0;
                bcs = 1;
            }
            if (s_abort) {
                // the MMA of tile i + 1 may be in flight: let it finish before leaving
                if (i + 1 < nT) {
                    mbar_wait_bounded(smem_u32(&s_mma[(i + 1) & 1]), (mphase >> ((i + 1) & 1)) & 1u, 1ll << 24);
                    mphase ^= (1u << ((i + 1) & 1));
                }
                break;
            }
        }
        if (resident) loaded_now = false;
        if (s_abort) break;

        // ---- uncertified searches of this warpgroup's grid: exact window search
        {
            unsigned mask = __ballot_sync(0xFFFFFFFFu, need);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                double z[DM];
                if (lane == src) exact_sample<DM>(p, s_pf, s_pd, k, ms, wg == 1, z);
                const int r = warp_window_nn<DM>(xown, Aown, z, src, p.rec32 + Gown.roff * Rec32<DM>::kFloats,
                                                 Gown.Npad, p.g64 + Gown.goff * d, Gown.N, d);
                if (lane == src) cown = r;
                if (lane == 0) atomicAdd(&p.status->rechecks, 1ull);
            }
        }
        if (wg == 1) s_mbc[t] = cown;     // hand cell j to warpgroup 0
        __syncthreads();

        // ---- counters p^k_ij
        if (wg == 0 && valid) {
            const int ci = cown, cj = s_mbc[t];
            if ((unsigned)ci >= (unsigned)L.NA || (unsigned)cj >= (unsigned)L.NB) {
                record_error(p.status, 6 /* QT_EDEVICE */, 13);
            } else {
                count_add(p.counts, p.counts_u32, L.coff + (long long)ci * L.NB + cj, 1u);
                if (p.cellsA) {
                    p.cellsA[ms] = ci;
                    p.cellsB[ms] = cj;
                }
                if (p.dump_count > 0 && (ms % (unsigned long long)p.dump_stride) == 0ull) {
                    const unsigned long long tt = ms / (unsigned long long)p.dump_stride;
                    if (tt < (unsigned long long)p.dump_count) {
                        const long long row = (long long)k * p.dump_count + (long long)tt;
                        double zx[DM], zy[DM];
                        exact_sample<DM>(p, s_pf, s_pd, k, ms, false, zx);
                        exact_sample<DM>(p, s_pf, s_pd, k, ms, true, zy);
                        for (int l = 0; l < d; ++l) {
                            p.dumpX[row * d + l] = zx[l];
                            p.dumpY[row * d + l] = zy[l];
                        }
                        p.dumpI[row] = ci;
                        p.dumpJ[row] = cj;
                    }
                }
            }
        }
        __syncthreads();
    }

    // ---- release the tensor memory (every MMA issued has completed: each was waited)
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(2 * kTcTileN))
                     : "memory");
    }
}

template <int DM, int KT>
static cudaError_t launch_tc(const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st)
{
    auto kern = forward_tc_kernel<DM, KT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, dyn);
    if (e != cudaSuccess) return e;
    if (b != 1) return cudaErrorInvalidConfiguration;   // one CTA per SM: it owns all 512 TMEM columns
    *bps = b;
    long long grid = (long long)num_sms * b;
    if (grid > p.total_items) grid = p.total_items;
    kern<<<(unsigned)grid, 256, dyn, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tc_forward(int dm, const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st)
{
    if (dm == 2) return launch_tc<2, 1>(p, dyn, num_sms, bps, st);
    if (dm == 4) return launch_tc<4, 1>(p, dyn, num_sms, bps, st);
    if (dm == 6) return launch_tc<6, 2>(p, dyn, num_sms, bps, st);
    if (dm == 8) return launch_tc<8, 2>(p, dyn, num_sms, bps, st);
    if (dm == 10) return launch_tc<10, 2>(p, dyn, num_sms, bps, st);
    return cudaErrorInvalidValue;
}

}  // namespace qt
