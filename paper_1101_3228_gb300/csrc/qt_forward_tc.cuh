// qt_forward_tc.cuh -- the forward step of Algorithm III (Pages & Wilbertz,
// arXiv:1101.3228, Sec. 4) with the nearest-cell screen on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// The screen scores s_j = |g_j|^2 - 2 x^.g_j (g_j, x^ centred on the grid's
// FP32 centre) are one GEMM per 128 samples x 256 grid points: sample rows
// [a_hi, a_hi, a_lo, 1, 1] times grid rows [g_hi, g_lo, g_hi, cc_hi, cc_lo],
// a = -2 sigma x^, g = sigma g^, cc = sigma^2 |g^|^2, each split into an FP16
// head and an FP16 tail, sigma = 2^tc_exp so that the grid fits in [-1, 1].
// Each group of coordinates takes DM columns (the dimension class, zero
// padded), so K = 16 holds 3 DM + 2 columns for DM <= 4 and K = 32 for
// DM <= 10.  The three cross products reproduce the FP32 score to about
// 2^-21 relative (the tail x tail product is below 2^-22).
//
// The screen kernel, one persistent CTA of 16 warps per SM over the work items
// (layer k, 128 samples each), in one of two layouts that the autotuner picks
// per dimension class by timing both:
//   DRAW_IN = true   the certifier warps draw every item's pairs into an item
//                    slot in shared memory: the whole step is one launch and
//                    the samples never touch device memory;
//   DRAW_IN = false  a separate high-occupancy draw pass (tc_draw_kernel)
//                    writes each item's operand rows and centred samples to
//                    device memory (up to 2 GiB per launch window), and warp 11
//                    copies them into the item slots with bulk copies.
// The roles of the screen kernel meet only at mbarriers:
//     two MMA warps        one per epilogue warpgroup; tile g of the CTA's
//                          sequence goes to warpgroup g & 1, its 256 points in
//                          kAccN-point slices to that warpgroup's kAccPerWg
//                          TMEM accumulators (512 columns in all);
//     a loader warp        bulk copies of the grids' operand tiles, kept for
//                          the whole layer when both grids fit, else streamed
//                          through a ring;
//     two epilogue         read their accumulators with tcgen05.ld.red (the
//     warpgroups           minimum of each 16-column chunk) and keep, per
//                          sample, the two best chunks and the smallest other
//                          chunk minimum;
//     four certifier       (draw,) merge the two warpgroups' chunk states,
//     warps                certify, recheck and count.
// While the tensor cores work on item n, the certifiers finish item n - 1.
//
// Exactness: the best chunk is re-scored on the CUDA cores in FP32 (and the
// second one when the certificate needs it), and the pick is certified against
// the exact FP64 distance with the FP32 bound inside the re-scored chunks and
// the tensor-core bound outside them; uncertified samples go to the exact
// window search (FP32 screen of the whole grid, exact FP64 distances inside
// the certified window).
#pragma once
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

// Minima of four consecutive 16-column chunks of this thread's accumulator row
// (columns taddr .. taddr + 63): tcgen05.ld.red loads 16 columns and returns
// their minimum; the loaded values themselves go to scratch registers local to
// this block, which also waits for the loads, so nothing outside it can touch
// registers the loads are still writing.
__device__ __forceinline__ void tc_chunk_min4(uint32_t taddr, float& m0, float& m1, float& m2, float& m3)
{
    asm volatile(
        "{\n\t.reg .f32 a<16>, b<16>, c<16>, e<16>;\n\t"
        "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 {a0,a1,a2,a3,a4,a5,a6,a7,a8,a9,a10,a11,a12,a13,a14,a15}, %0, [%4];\n\t"
        "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 {b0,b1,b2,b3,b4,b5,b6,b7,b8,b9,b10,b11,b12,b13,b14,b15}, %1, [%5];\n\t"
        "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 {c0,c1,c2,c3,c4,c5,c6,c7,c8,c9,c10,c11,c12,c13,c14,c15}, %2, [%6];\n\t"
        "tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 {e0,e1,e2,e3,e4,e5,e6,e7,e8,e9,e10,e11,e12,e13,e14,e15}, %3, [%7];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t}"
        : "=f"(m0), "=f"(m1), "=f"(m2), "=f"(m3)
        : "r"(taddr), "r"(taddr + 16u), "r"(taddr + 32u), "r"(taddr + 48u)
        : "memory");
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
// All 16 records are loaded before any of them is compared, so that their
// loads are in flight together.
template <int DM>
__device__ __forceinline__ void cc_chunk(const float* __restrict__ recs, int chunk, const float (&x)[DM], int& idx,
                                         float& best, float& S1, float& r1)
{
    constexpr int F = Rec32<DM>::kFloats;
    constexpr int V = F / 4;
    const float4* r4 = reinterpret_cast<const float4*>(recs) + (long long)chunk * kChunk * V;
    float sc[kChunk];
#pragma unroll
    for (int q = 0; q < kChunk; ++q) {
        float4 a[V];
#pragma unroll
        for (int v = 0; v < V; ++v) a[v] = r4[q * V + v];
        float f[4 * V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            f[4 * v] = a[v].x;
            f[4 * v + 1] = a[v].y;
            f[4 * v + 2] = a[v].z;
            f[4 * v + 3] = a[v].w;
        }
        float s = f[0];
#pragma unroll
        for (int l = 0; l < DM; ++l) s = __fmaf_rn(x[l], f[1 + l], s);
        sc[q] = s;
    }
    best = sc[0];
    S1 = __int_as_float(0x7F800000);
    int bq = 0;
#pragma unroll
    for (int q = 1; q < kChunk; ++q) {
        const bool t = sc[q] < best;
        S1 = fminf(S1, t ? best : sc[q]);
        best = t ? sc[q] : best;
        bq = t ? q : bq;
    }
    idx = chunk * kChunk + bq;
    const float* r = recs + (long long)idx * F;
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


__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait with one outcome for the whole warp (the epilogue's tcgen05.ld
// and the certifiers' ballots need converged warps).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, long long budget)
{
    const bool ok = mbar_wait_bounded(bar, parity, budget);
    return __all_sync(0xFFFFFFFFu, ok);
}

__device__ __forceinline__ int layer_of(const ForwardParams& p, long long item)
{
    int lo = 0, hi = p.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.layers[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per sample, over the chunks a warpgroup has seen (in increasing order): the
// best chunk minimum B1 (chunk bc), the second Bs (chunk bcs) and the smallest
// of the others B3; ties keep the lower chunk.
struct ChunkTrack {
    float B1, Bs, B3;
    int bc, bcs;
    __device__ __forceinline__ void reset()
    {
        B1 = Bs = B3 = __int_as_float(0x7F800000);
        bc = 0;
        bcs = 1;
    }
    __device__ __forceinline__ void add(float mc, int c)
    {
        const bool t1 = mc < B1, t2 = mc < Bs;
        B3 = fminf(B3, fmaxf(mc, Bs));
        Bs = fminf(Bs, fmaxf(mc, B1));
        bcs = t1 ? bc : (t2 ? c : bcs);
        B1 = fminf(B1, mc);
        bc = t1 ? c : bc;
    }
};

__device__ __forceinline__ bool pair_less(float a, int ia, float b, int ib)
{
    return a < b || (a == b && ia < ib);
}

__device__ __forceinline__ void pair_sort2(float& a, int& ia, float& b, int& ib)
{
    if (pair_less(b, ib, a, ia)) {
        const float v = a;
        a = b;
        b = v;
        const int i = ia;
        ia = ib;
        ib = i;
    }
}

}  // namespace



namespace {

constexpr int kEpiWarps = 8;       // warps 0-7: epilogue warpgroups 0 and 1
constexpr int kMmaWarp0 = 8;       // warps 8, 9: MMAs for epilogue warpgroups 0, 1
constexpr int kLoadWarp = 10;      // warp 10: bulk copies of the operand tiles
constexpr int kOpWarp = 11;        // warp 11: bulk copies of each item's drawn samples (draw pass layout)
constexpr int kCertWarp0 = 12;     // warps 12-15: (draw,) certify, recheck, count
constexpr int kAccN = 256;             // columns of one accumulator (MMA N): a whole tile
constexpr int kAccPerWg = kTcTileN / kAccN;   // accumulators per epilogue warpgroup (one tile)
constexpr int kAccs = 2 * kAccPerWg;   // 512 TMEM columns in all
static_assert(kAccs * kAccN == 2 * kTcTileN && kAccN % 64 == 0, "accumulator layout");
static_assert(kTcThreads == 16 * 32, "role layout");

// What a certifier warp needs of the layer of an item (shared memory, one per
// warp and operand slot, plus one for the layer of its draws).
struct SlotLayer {
    long long item_begin, coff, goffA, goffB, roffA, roffB;
    int32_t k, NA, NB, NpadA, NpadB, expA, expB, spare;
};

}  // namespace

// Draw of one work item's sample row t (Algorithm III: the pair (X_k, X_{k+1})
// of the AR(1) step), straight into the item slot in shared memory: the FP16 operand rows of both grids
// ([a_hi (DM), a_hi (DM), a_lo (DM), 1, 1], a = -2 sigma (x - mu), core-matrix
// layout, K columns) and the centred FP32 coordinates with their norm (sign bit
// set when a coordinate leaves the FP16 range).  Parameters and grid centres
// are read from global memory (the same addresses for every thread: broadcast
// loads that stay in L1).
template <int DM, int K>
__device__ __forceinline__ void draw_row(const ForwardParams& p, int k, const LayerDesc& L, unsigned long long m,
                                         int t, unsigned char* ops_slot, float* cert_slot)
{
    constexpr int kOpBytes = kTcTileM * K * 2;
    const int d = p.d;
    const GridInfo& GA = p.grids[L.gridA];
    const GridInfo& GB = p.grids[L.gridB];
    float muA[DM], muB[DM];
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        muA[l] = GA.mu[l];
        muB[l] = GB.mu[l];
    }
    const float* spf = p.params_f ? p.params_f + (long long)k * p.params_stride : nullptr;
    const double* spd = p.params_d ? p.params_d + (long long)k * p.params_stride : nullptr;
    const Centred<DM> cs = centred_sample_inl<DM>(p, spf, spd, muA, muB, k, m);
#pragma unroll
    for (int gr = 0; gr < 2; ++gr) {
        const float* x = gr == 0 ? cs.xa : cs.yb;
        const float A = gr == 0 ? cs.Aa : cs.Ab;
        const float sg = ldexpf(1.0f, gr == 0 ? GA.tc_exp : GB.tc_exp);
        bool big = false;
#pragma unroll
        for (int l = 0; l < DM; ++l)
            if (l < d) big = big || !(fabsf(sg * x[l]) <= 16384.0f);
        uint32_t hi[DM], lo[DM];
#pragma unroll
        for (int l = 0; l < DM; ++l) {
            const float v = (l < d && !big) ? sg * x[l] : 0.0f;
            const __half h = __float2half_rn(v);
            hi[l] = __half_as_ushort(h);
            lo[l] = __half_as_ushort(__float2half_rn(v - __half2float(h)));
        }
        const uint32_t one = __half_as_ushort(__float2half_rn(1.0f));
        uint32_t w[K / 2];
#pragma unroll
        for (int q = 0; q < K; q += 2) {
            uint32_t h2[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int c = q + u;
                h2[u] = c < DM ? hi[c] : (c < 2 * DM ? hi[c - DM] : (c < 3 * DM ? lo[c - 2 * DM] : (c < 3 * DM + 2 ? one : 0u)));
            }
            w[q / 2] = h2[0] | (h2[1] << 16);
        }
        unsigned char* base = ops_slot + gr * kOpBytes;
#pragma unroll
        for (int kb = 0; kb < K / 8; ++kb)
            *reinterpret_cast<uint4*>(base + (((t >> 3) * (K / 8) + kb) * 64 + (t & 7) * 8) * 2) =
                make_uint4(w[4 * kb], w[4 * kb + 1], w[4 * kb + 2], w[4 * kb + 3]);
        float* cx = cert_slot + gr * (DM + 1) * kTcTileM + t;
#pragma unroll
        for (int l = 0; l < DM; ++l) cx[l * kTcTileM] = x[l];
        cx[DM * kTcTileM] = __int_as_float(__float_as_int(A) | (big ? (int)0x80000000 : 0));
    }
}

template <int DM, int KT, bool DRAW_IN>
__global__ void __launch_bounds__(kTcThreads, 1) forward_tc_kernel(const ForwardParams p)
{
    constexpr int K = 16 * KT;
    static_assert(3 * DM + 2 <= K, "operand row");
    constexpr int kTileBytes = kTcTileN * K * 2;
    constexpr int kOpBytes = kTcTileM * K * 2;
    constexpr int F = Rec32<DM>::kFloats;
    const float kInf = __int_as_float(0x7F800000);
    extern __shared__ __align__(128) unsigned char dsm_tc[];
    __shared__ __align__(8) unsigned long long s_tfull[kTcMaxSlots], s_tempty[kTcMaxSlots];
    __shared__ __align__(8) unsigned long long s_accfull[kAccs], s_accempty[kAccs];
    __shared__ __align__(8) unsigned long long s_opfull[2], s_opempty[2];
    __shared__ __align__(8) unsigned long long s_stA[2], s_stB[2], s_stempty[2];
    __shared__ __align__(8) unsigned long long s_drain[2], s_ldone;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ SlotLayer s_slot[4][2];
    __shared__ __align__(8) unsigned long long s_certdone[2];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int d = p.d;
    const int RS = p.tc_slots;
    const long long G = gridDim.x;
    // dynamic shared memory: [tile ring][sample operands][chunk states][centred samples][parameters]
    unsigned char* ring = dsm_tc;
    unsigned char* ops = ring + (size_t)RS * kTileBytes;                       // [item slot][grid] rows
    float* sst = reinterpret_cast<float*>(ops + 4 * kOpBytes);                 // [slot][grid][wg][5][128]
    float* scert = sst + 2 * 2 * 2 * 5 * kTcTileM;                             // [slot][grid][DM + 1][128]
    constexpr long long kItemOp = tc_item_op_bytes(K), kItemCert = tc_item_cert_bytes(DM);
    static_assert(kItemOp == 2 * kOpBytes && kItemCert == 2 * (DM + 1) * kTcTileM * 4, "item layout");
    const uint32_t ring_u = smem_u32(ring), ops_u = smem_u32(ops);

    if (tid == 0) {
        for (int i = 0; i < kTcMaxSlots; ++i) {
            mbar_init(smem_u32(&s_tfull[i]), 1);
            mbar_init(smem_u32(&s_tempty[i]), 1);
        }
        for (int a = 0; a < kAccs; ++a) {
            mbar_init(smem_u32(&s_accfull[a]), 1);
            mbar_init(smem_u32(&s_accempty[a]), 128);
        }
        for (int b = 0; b < 2; ++b) {
            // filled by the certifier threads' draws, or by the bulk copies of the draw pass
            mbar_init(smem_u32(&s_opfull[b]), DRAW_IN ? 128 : 1);
            mbar_init(smem_u32(&s_opempty[b]), 2);    // the two MMA warps' commits
            mbar_init(smem_u32(&s_certdone[b]), 128); // the certifier threads, done with the slot
            mbar_init(smem_u32(&s_stA[b]), 256);
            mbar_init(smem_u32(&s_stB[b]), 256);
            mbar_init(smem_u32(&s_stempty[b]), 128);
        }
        mbar_init(smem_u32(&s_drain[0]), 1);
        mbar_init(smem_u32(&s_drain[1]), 1);
        mbar_init(smem_u32(&s_ldone), 2);
        s_abort = 0;
        fence_proxy_async();
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
    volatile int* abort_flag = &s_abort;

    if (warp == kMmaWarp0 || warp == kMmaWarp0 + 1) {
        // ================================================================ MMAs
        // tile g of the CTA's sequence goes to warpgroup g & 1, which has its
        // own issuing warp; slice h of the tile (kAccN points) goes to that
        // warpgroup's accumulator kAccPerWg (g & 1) + h
        const int ib = warp - kMmaWarp0;
        if (lane == 0) {
            const bool resident = p.tc_resident != 0;
            const uint32_t idesc = (1u << 4) | ((uint32_t)(kAccN >> 3) << 17) | ((uint32_t)(kTcTileM >> 4) << 24);
            int tA = 0, nT = 0, layers = 0, lastT = 0;
            long long lbeg = 0, lend = 0;
            uint32_t tph = 0, pend = 0;        // resident: parity of each slot's current load, slots not yet waited
            int rslot = ib;                    // streamed: ring slot and parity of this warp's next tile
            uint32_t rph = 0;
            if (!resident && rslot >= RS) {
                rslot -= RS;
                rph = 1;
            }
            long long g = 0;                   // tiles of the CTA's sequence so far
            bool ok = true;
            auto fail = [&](int where) {
                record_error(p.status, 4 /* QT_ETIMEOUT */, where);
                *abort_flag = 1;
                ok = false;
            };
            for (long long n = 0; ok; ++n) {
                const long long item = p.item_lo + blockIdx.x + n * G;
                if (item >= p.item_hi || *abort_flag) break;
                if (item < lbeg || item >= lend) {
                    const LayerDesc& L = p.layers[layer_of(p, item)];
                    lbeg = L.item_begin;
                    lend = lbeg + L.items;
                    tA = p.grids[L.gridA].tc_tiles;
                    nT = tA + p.grids[L.gridB].tc_tiles;
                    if (resident) {
                        // the loader overwrites the tiles once both warps' MMAs of the previous layer are done
                        if (layers > 0) {
                            tc_commit(smem_u32(&s_ldone));
                            for (int i = 0; i < lastT; ++i) tph ^= 1u << i;
                        }
                        pend = nT >= 32 ? ~0u : ((1u << nT) - 1u);
                        lastT = nT;
                    }
                    ++layers;
                }
                const int os = (int)(n & 1);
                if (!mbar_wait_bounded(smem_u32(&s_opfull[os]), (uint32_t)((n >> 1) & 1), p.spin_budget)) {
                    fail(22);
                    break;
                }
                for (int i = (int)((g & 1) ^ (long long)ib); i < nT && ok; i += 2) {
                    const long long gg = g + i;
                    int slot;
                    if (resident) {
                        slot = i;
                        if ((pend >> i) & 1u) {
                            if (!mbar_wait_bounded(smem_u32(&s_tfull[i]), (tph >> i) & 1u, p.spin_budget)) {
                                fail(24);
                                break;
                            }
                            pend &= ~(1u << i);
                        }
                    } else {
                        slot = rslot;
                        if (!mbar_wait_bounded(smem_u32(&s_tfull[slot]), rph, p.spin_budget)) {
                            fail(24);
                            break;
                        }
                    }
                    const uint32_t a_base = ops_u + (uint32_t)((os * 2 + (i < tA ? 0 : 1)) * kOpBytes);
#pragma unroll
                    for (int h = 0; h < kAccPerWg; ++h) {
                        const int acc = kAccPerWg * ib + h;
                        if (!mbar_wait_bounded(smem_u32(&s_accempty[acc]), (uint32_t)((gg >> 1) & 1) ^ 1u,
                                               p.spin_budget)) {
                            fail(23);
                            break;
                        }
                        tc_fence_after();
                        // rows 128h .. 128h + 127 of the tile: 16 row blocks of K * 16 bytes further
                        const uint32_t b_base = ring_u + (uint32_t)(slot * kTileBytes + h * (kAccN / 8) * K * 16);
                        const uint32_t dt = tmem + (uint32_t)(acc * kAccN);
#pragma unroll
                        for (int s = 0; s < KT; ++s) {
                            const uint64_t ad = smem_desc(a_base + s * 256, 128, K * 16);
                            const uint64_t bd = smem_desc(b_base + s * 256, 128, K * 16);
                            tc_mma(dt, ad, bd, idesc, s > 0 ? 1u : 0u);
                        }
                        tc_commit(smem_u32(&s_accfull[acc]));
                    }
                    if (ok && !resident) {
                        tc_commit(smem_u32(&s_tempty[slot]));
                        rslot += 2;
                        if (rslot >= RS) {
                            rslot -= RS;
                            rph ^= 1u;
                        }
                    }
                }
                if (!ok) break;
                tc_commit(smem_u32(&s_opempty[os]));
                g += nT;
            }
            // every MMA issued completes before the tensor memory is released
            tc_commit(smem_u32(&s_drain[ib]));
            mbar_wait_bounded(smem_u32(&s_drain[ib]), 0u, kDrainUs);
        }
    } else if (warp == kLoadWarp) {
        // ================================================================ operand tiles
        if (lane == 0) {
            const bool resident = p.tc_resident != 0;
            const unsigned char* tiles = reinterpret_cast<const unsigned char*>(p.tc_tiles);
            long long lbeg = 0, lend = 0, toffA = 0, toffB = 0;
            int tA = 0, nT = 0;
            auto refresh = [&](long long item) {
                const LayerDesc& L = p.layers[layer_of(p, item)];
                lbeg = L.item_begin;
                lend = lbeg + L.items;
                tA = p.grids[L.gridA].tc_tiles;
                nT = tA + p.grids[L.gridB].tc_tiles;
                toffA = p.grids[L.gridA].tc_toff;
                toffB = p.grids[L.gridB].tc_toff;
            };
            auto copy = [&](int slot, int i) {
                const long long src = i < tA ? toffA + i : toffB + (i - tA);
                mbar_arrive_expect_tx(smem_u32(&s_tfull[slot]), kTileBytes);
                bulk_g2s(ring_u + slot * kTileBytes, tiles + src * kTileBytes, kTileBytes, smem_u32(&s_tfull[slot]));
            };
            auto fail = [&](int where) {
                record_error(p.status, 4 /* QT_ETIMEOUT */, where);
                *abort_flag = 1;
            };
            if (resident) {
                // all tiles of a layer pair, once per layer
                int layers = 0, lastT = 0;
                uint32_t tph = 0;              // per slot: parity of the next load's completion
                for (long long n = 0;; ++n) {
                    const long long item = p.item_lo + blockIdx.x + n * G;
                    if (item >= p.item_hi || *abort_flag) break;
                    if (item >= lbeg && item < lend) continue;
                    refresh(item);
                    if (layers > 0 &&
                        !mbar_wait_bounded(smem_u32(&s_ldone), (uint32_t)((layers - 1) & 1), p.spin_budget)) {
                        fail(21);
                        break;
                    }
                    if (layers > 0)
                        for (int i = 0; i < lastT; ++i) tph ^= 1u << i;
                    for (int i = 0; i < nT; ++i) copy(i, i);
                    lastT = nT;
                    ++layers;
                }
                // the last layer's copies land before the shared memory is released
                for (int i = 0; i < lastT; ++i) mbar_wait_bounded(smem_u32(&s_tfull[i]), (tph >> i) & 1u, kDrainUs);
            } else {
                // the tiles of every item in order, through the ring
                long long ql = 0, ln = 0;
                int li = 0, r = 0;
                uint32_t rph = 0;              // parity of the ring's current lap
                while (true) {
                    const long long item = p.item_lo + blockIdx.x + ln * G;
                    if (item >= p.item_hi || *abort_flag) break;
                    if (li == 0 && (item < lbeg || item >= lend)) refresh(item);
                    if (!mbar_wait_bounded(smem_u32(&s_tempty[r]), rph ^ 1u, p.spin_budget)) {
                        fail(25);
                        break;
                    }
                    copy(r, li);
                    ++ql;
                    if (++r == RS) {
                        r = 0;
                        rph ^= 1u;
                    }
                    if (++li == nT) {
                        li = 0;
                        ++ln;
                    }
                }
                // the copies of the last lap land before the shared memory is released
                for (int q = 0; q < RS && q < ql; ++q) {
                    if (--r < 0) {
                        r = RS - 1;
                        rph ^= 1u;
                    }
                    mbar_wait_bounded(smem_u32(&s_tfull[r]), rph, kDrainUs);
                }
            }
        }
    } else if (warp < kEpiWarps) {
        // ================================================================ epilogue
        const int wg = warp >> 2;
        const int t = (warp & 3) * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        int tA = 0, nT = 0;
        long long g = 0, lbeg = 0, lend = 0;
        ChunkTrack tr;
        auto process = [&](long long gg, int lt) -> bool {
#pragma unroll
            for (int h = 0; h < kAccPerWg; ++h) {
                const int acc = kAccPerWg * wg + h;
                if (!warp_wait(smem_u32(&s_accfull[acc]), (uint32_t)((gg >> 1) & 1), p.spin_budget)) return false;
                tc_fence_after();
                // all chunk minima of the accumulator first, so that it goes back to
                // the MMA warp before the tracking work
                float mc[kAccN / kChunk];
#pragma unroll
                for (int q = 0; q < kAccN / 64; ++q)
                    tc_chunk_min4(trow + (uint32_t)(acc * kAccN + q * 64), mc[4 * q], mc[4 * q + 1], mc[4 * q + 2],
                                  mc[4 * q + 3]);
                tc_fence_before();
                mbar_arrive(smem_u32(&s_accempty[acc]));
                const int c0 = lt * (kTcTileN / kChunk) + h * (kAccN / kChunk);
#pragma unroll
                for (int q = 0; q < kAccN / kChunk; ++q) tr.add(mc[q], c0 + q);
            }
            return true;
        };
        auto dump = [&](int s, int gr) {
            float* st = sst + ((s * 2 + gr) * 2 + wg) * 5 * kTcTileM + t;
            st[0 * kTcTileM] = tr.B1;
            st[1 * kTcTileM] = tr.Bs;
            st[2 * kTcTileM] = tr.B3;
            st[3 * kTcTileM] = __int_as_float(tr.bc);
            st[4 * kTcTileM] = __int_as_float(tr.bcs);
        };
        for (long long n = 0;; ++n) {
            const long long item = p.item_lo + blockIdx.x + n * G;
            if (item >= p.item_hi) break;
            if (__shfl_sync(0xFFFFFFFFu, *abort_flag, 0)) break;
            if (item < lbeg || item >= lend) {
                const LayerDesc& L = p.layers[layer_of(p, item)];
                lbeg = L.item_begin;
                lend = lbeg + L.items;
                tA = p.grids[L.gridA].tc_tiles;
                nT = tA + p.grids[L.gridB].tc_tiles;
            }
            const int s = (int)(n & 1);
            bool ok = true;
            // grid A: tiles i < tA with (g + i) & 1 == wg
            tr.reset();
            for (int i = (int)((g & 1) ^ wg); ok && i < tA; i += 2) ok = process(g + i, i);
            if (ok) ok = warp_wait(smem_u32(&s_stempty[s]), (uint32_t)((n >> 1) & 1) ^ 1u, p.spin_budget);
            if (ok) {
                dump(s, 0);
                mbar_arrive(smem_u32(&s_stA[s]));
            }
            // grid B
            tr.reset();
            for (int i = tA + (int)(((g + tA) & 1) ^ wg); ok && i < nT; i += 2) ok = process(g + i, i - tA);
            if (ok) {
                dump(s, 1);
                mbar_arrive(smem_u32(&s_stB[s]));
            }
            if (!ok) {
                if (lane == 0) {
                    record_error(p.status, 4 /* QT_ETIMEOUT */, 26);
                    *abort_flag = 1;
                }
                break;
            }
            g += nT;
        }
    } else if (warp == kOpWarp) {
        // ================================================================ drawn samples (draw pass)
        // item n's operand rows and centred samples, as the draw pass wrote them,
        // go to slot n & 1 once the MMAs and the certifiers are done with item n - 2
        if constexpr (!DRAW_IN) {
            if (lane == 0) {
                long long n = 0;
                for (;; ++n) {
                    const long long item = p.item_lo + blockIdx.x + n * G;
                    if (item >= p.item_hi || *abort_flag) break;
                    const int s = (int)(n & 1);
                    const uint32_t par = (uint32_t)((n >> 1) & 1) ^ 1u;
                    if (!mbar_wait_bounded(smem_u32(&s_opempty[s]), par, p.spin_budget) ||
                        !mbar_wait_bounded(smem_u32(&s_certdone[s]), par, p.spin_budget)) {
                        record_error(p.status, 4 /* QT_ETIMEOUT */, 27);
                        *abort_flag = 1;
                        break;
                    }
                    const unsigned char* src = p.tc_items + (item - p.item_lo) * (kItemOp + kItemCert);
                    const uint32_t bar = smem_u32(&s_opfull[s]);
                    mbar_arrive_expect_tx(bar, (uint32_t)(kItemOp + kItemCert));
                    bulk_g2s(ops_u + (uint32_t)(s * kItemOp), src, (uint32_t)kItemOp, bar);
                    bulk_g2s(smem_u32(scert) + (uint32_t)(s * kItemCert), src + kItemOp, (uint32_t)kItemCert, bar);
                }
                // the copies of the last two items land before the shared memory is released
                for (long long q = n > 2 ? n - 2 : 0; q < n; ++q)
                    mbar_wait_bounded(smem_u32(&s_opfull[q & 1]), (uint32_t)((q >> 1) & 1), kDrainUs);
            }
        }
    } else if (warp >= kCertWarp0) {
        // ================================================================ certifiers
        const int cw = warp - kCertWarp0;
        const int t = cw * 32 + lane;
        SlotLayer* sl = s_slot[cw];               // layer of the item in each slot
        long long lbeg = 0, lend = 0;
        SlotLayer cur;
        cur.k = -1;
        int slot_k[2] = {-1, -1};
        auto fail = [&](int where) {
            if (lane == 0) {
                record_error(p.status, 4 /* QT_ETIMEOUT */, where);
                *abort_flag = 1;
            }
        };
        // Merge the warpgroups' chunk states of row t, re-score the best chunk
        // in FP32 and try the certificate (first pass, straight-line code, so
        // that the two grids' passes overlap); then, where the certificate
        // needs it, re-score the second chunk too and finish.
        struct Pass {
            float x[DM];
            float A, rest, v1, inv_sg, best, in2, r1;
            int idx, mbc, c1, nch, why;
            bool big, chunk_ok, tcok;
            const float* recs;
        };
        auto first = [&](int s, int gr, const SlotLayer& S, Pass& c) {
            const int Npad = gr == 0 ? S.NpadA : S.NpadB;
            const float* st = sst + (s * 2 + gr) * 2 * 5 * kTcTileM + t;
            float v0 = st[0], v1 = st[kTcTileM], v2 = st[5 * kTcTileM], v3 = st[6 * kTcTileM];
            int c0 = __float_as_int(st[3 * kTcTileM]), c1 = __float_as_int(st[4 * kTcTileM]);
            int c2 = __float_as_int(st[8 * kTcTileM]), c3 = __float_as_int(st[9 * kTcTileM]);
            float rest = fminf(st[2 * kTcTileM], st[7 * kTcTileM]);
            pair_sort2(v0, c0, v1, c1);
            pair_sort2(v2, c2, v3, c3);
            pair_sort2(v0, c0, v2, c2);
            pair_sort2(v1, c1, v3, c3);
            pair_sort2(v1, c1, v2, c2);
            c.rest = fminf(rest, fminf(v2, v3));
            c.v1 = v1;
            c.c1 = c1;
            c.nch = Npad / kChunk;
            const float* cx = scert + (s * 2 + gr) * (DM + 1) * kTcTileM + t;
#pragma unroll
            for (int l = 0; l < DM; ++l) c.x[l] = cx[l * kTcTileM];
            const float Araw = cx[DM * kTcTileM];
            c.big = (__float_as_int(Araw) & (int)0x80000000) != 0;
            c.A = fabsf(Araw);
            c.inv_sg = ldexpf(1.0f, -(gr == 0 ? S.expA : S.expB));
            c.recs = p.rec32 + (gr == 0 ? S.roffA : S.roffB) * F;
            c.chunk_ok = c0 >= 0 && c0 < c.nch;
            c.mbc = c.chunk_ok ? c0 : 0;
        };
        // the FP32 re-score of the best chunk (records from L2) and the certificate
        auto score = [&](Pass& c) {
            cc_chunk<DM>(c.recs, c.mbc, c.x, c.idx, c.best, c.in2, c.r1);
            // FP32 inside the best chunk, tensor-core scores outside it
            c.why = 0;
            c.tcok = tc_certified(d, c.A, c.best, c.in2, fminf(c.v1, c.rest) * c.inv_sg * c.inv_sg, c.r1, c.inv_sg,
                                  c.why);
        };
        auto finish = [&](Pass& c, int Nown, bool valid, bool& need) -> int {
            if (!c.tcok && c.why == 2 && c.c1 >= 0 && c.c1 < c.nch && c.c1 != c.mbc) {
                // the second chunk competes: FP32 inside both, tensor-core scores outside
                int idx2;
                float best2, S12, r12;
                cc_chunk<DM>(c.recs, c.c1, c.x, idx2, best2, S12, r12);
                if (best2 < c.best || (best2 == c.best && idx2 < c.idx)) {
                    c.in2 = fminf(S12, c.best);
                    c.best = best2;
                    c.idx = idx2;
                    c.r1 = r12;
                } else {
                    c.in2 = fminf(c.in2, best2);
                }
                c.tcok = tc_certified(d, c.A, c.best, c.in2, c.rest * c.inv_sg * c.inv_sg, c.r1, c.inv_sg, c.why);
            }
            const bool rng_ok = c.chunk_ok && c.idx < Nown && !c.big;
            const bool cert = c.tcok && rng_ok;
            if (valid && !cert) atomicAdd(&p.status->spare[!rng_ok ? 3 : c.why], 1ull);
            need = valid && !cert;
            return c.idx;
        };
        // exact window search of the lanes in `need` (the whole warp takes part),
        // from the centred sample the first pass copied out of the item slot
        auto recheck = [&](const Pass& c, int gr, const SlotLayer& S, unsigned long long ms, bool need, int& cell) {
            unsigned mask = __ballot_sync(0xFFFFFFFFu, need);
            if (!mask) return;
            const float A = c.A;
            const int k = S.k;
            const float* gpf = p.params_f ? p.params_f + (long long)k * p.params_stride : nullptr;
            const double* gpd = p.params_d ? p.params_d + (long long)k * p.params_stride : nullptr;
            const float* recs = p.rec32 + (gr == 0 ? S.roffA : S.roffB) * F;
            const double* g64 = p.g64 + (gr == 0 ? S.goffA : S.goffB) * d;
            const int Npad = gr == 0 ? S.NpadA : S.NpadB;
            const int Nown = gr == 0 ? S.NA : S.NB;
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                double z[DM];
                if (lane == src) exact_sample<DM>(p, gpf, gpd, k, ms, gr == 1, z);
                const int r = warp_window_nn<DM>(c.x, A, z, src, recs, Npad, g64, Nown, d);
                if (lane == src) cell = r;
                if (lane == 0) atomicAdd(&p.status->rechecks, 1ull);
            }
        };
        // DRAW_IN: thread t draws sample row t of item nn of this CTA's sequence
        // into slot nn & 1 (items 0 and 1 first, item n + 2 once item n is
        // certified and its MMAs are complete); the generic-proxy stores are
        // fenced for the tensor cores' async-proxy reads before the MMA warps
        // are released
        long long dbeg = 0, dend = 0;
        int dk = 0;
        auto draw = [&](long long nn) {
            const long long item = p.item_lo + blockIdx.x + nn * G;
            if (item < dbeg || item >= dend) {
                dk = layer_of(p, item);
                dbeg = p.layers[dk].item_begin;
                dend = dbeg + p.layers[dk].items;
            }
            const unsigned long long mtile = (unsigned long long)(item - dbeg) * kTcTileM;
            const unsigned long long m = mtile + (unsigned long long)t;
            const int sl = (int)(nn & 1);
            draw_row<DM, K>(p, dk, p.layers[dk], m < p.M ? m : mtile, t, ops + sl * kItemOp,
                            scert + sl * 2 * (DM + 1) * kTcTileM);
            fence_proxy_async();
            mbar_arrive(smem_u32(&s_opfull[sl]));
        };
        if constexpr (DRAW_IN) {
            for (long long nn = 0; nn < 2; ++nn)
                if (p.item_lo + blockIdx.x + nn * G < p.item_hi) draw(nn);
        }
        for (long long n = 0;; ++n) {
            const long long item = p.item_lo + blockIdx.x + n * G;
            if (item >= p.item_hi) break;
            if (__shfl_sync(0xFFFFFFFFu, *abort_flag, 0)) break;
            const int s = (int)(n & 1);
            if (item < lbeg || item >= lend) {
                const int k = layer_of(p, item);
                const LayerDesc& L = p.layers[k];
                const GridInfo& GA = p.grids[L.gridA];
                const GridInfo& GB = p.grids[L.gridB];
                cur.item_begin = L.item_begin;
                cur.coff = L.coff;
                cur.goffA = GA.goff;
                cur.goffB = GB.goff;
                cur.roffA = GA.roff;
                cur.roffB = GB.roff;
                cur.k = k;
                cur.NA = L.NA;
                cur.NB = L.NB;
                cur.NpadA = GA.Npad;
                cur.NpadB = GB.Npad;
                cur.expA = GA.tc_exp;
                cur.expB = GB.tc_exp;
                lbeg = L.item_begin;
                lend = lbeg + L.items;
            }
            if (slot_k[s] != cur.k) {
                __syncwarp();
                if (lane == 0) sl[s] = cur;
                __syncwarp();
                slot_k[s] = cur.k;
            }
            const SlotLayer& S = sl[s];
            const unsigned long long ms = (unsigned long long)(item - S.item_begin) * kTcTileM + (unsigned long long)t;
            const bool valid = ms < p.M;
            bool needA = false, needB = false;
            // the centred samples of this item have landed (the MMAs waited for them too)
            if (!DRAW_IN && !warp_wait(smem_u32(&s_opfull[s]), (uint32_t)((n >> 1) & 1), p.spin_budget)) {
                fail(30);
                break;
            }
            if (!warp_wait(smem_u32(&s_stA[s]), (uint32_t)((n >> 1) & 1), p.spin_budget)) {
                fail(28);
                break;
            }
            if (!warp_wait(smem_u32(&s_stB[s]), (uint32_t)((n >> 1) & 1), p.spin_budget)) {
                fail(29);
                break;
            }
            Pass pa, pb;
            first(s, 0, S, pa);
            first(s, 1, S, pb);
            // the chunk states and the item slot are read (the passes hold copies):
            // release them before the L2 loads of the re-score, so that the epilogue
            // and the next item can move in
            mbar_arrive(smem_u32(&s_stempty[s]));
            if constexpr (!DRAW_IN) mbar_arrive(smem_u32(&s_certdone[s]));   // the draw pass may refill the slot
            score(pa);
            score(pb);
            int ci = finish(pa, S.NA, valid, needA);
            int cj = finish(pb, S.NB, valid, needB);
            recheck(pa, 0, S, ms, needA, ci);
            recheck(pb, 1, S, ms, needB, cj);
            if constexpr (DRAW_IN) {
                // item n + 2 into this slot, once item n is certified and its MMAs are
                // complete (drawing before the recheck keeps both passes' registers
                // live across the draw and spills more)
                if (p.item_lo + blockIdx.x + (n + 2) * G < p.item_hi) {
                    if (!warp_wait(smem_u32(&s_opempty[s]), (uint32_t)((n >> 1) & 1), p.spin_budget)) {
                        fail(31);
                        break;
                    }
                    draw(n + 2);
                }
            }
            // ---- counters p^k_ij
            if (valid) {
                if ((unsigned)ci >= (unsigned)S.NA || (unsigned)cj >= (unsigned)S.NB) {
                    record_error(p.status, 6 /* QT_EDEVICE */, 13);
                } else {
                    count_add(p.counts, p.counts_u32, S.coff + (long long)ci * S.NB + cj, 1u);
                    if (p.cellsA) {
                        p.cellsA[ms] = ci;
                        p.cellsB[ms] = cj;
                    }
                    if (p.dump_count > 0 && (ms % (unsigned long long)p.dump_stride) == 0ull) {
                        const unsigned long long tt = ms / (unsigned long long)p.dump_stride;
                        if (tt < (unsigned long long)p.dump_count) {
                            const int k = S.k;
                            const long long row = (long long)k * p.dump_count + (long long)tt;
                            const float* gpf = p.params_f ? p.params_f + (long long)k * p.params_stride : nullptr;
                            const double* gpd = p.params_d ? p.params_d + (long long)k * p.params_stride : nullptr;
                            double zx[DM], zy[DM];
                            exact_sample<DM>(p, gpf, gpd, k, ms, false, zx);
                            exact_sample<DM>(p, gpf, gpd, k, ms, true, zy);
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
        }
    }

    // ---- every role is done; the producer has drained the MMAs and copies
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(2 * kTcTileN))
                     : "memory");
    }
}

template <int DM, int KT, bool DRAW_IN>
cudaError_t launch_tc(const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st)
{
    auto kern = forward_tc_kernel<DM, KT, DRAW_IN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kTcThreads, dyn);
    if (e != cudaSuccess) return e;
    if (b != 1) return cudaErrorInvalidConfiguration;   // one CTA per SM: it owns all 512 TMEM columns
    if (p.tc_slots < 2 || p.tc_slots > kTcMaxSlots) return cudaErrorInvalidValue;
    *bps = b;
    long long grid = (long long)num_sms * b;
    if (grid > p.item_hi - p.item_lo) grid = p.item_hi - p.item_lo;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kTcThreads, dyn, st>>>(p);
    return cudaGetLastError();
}

}  // namespace qt
