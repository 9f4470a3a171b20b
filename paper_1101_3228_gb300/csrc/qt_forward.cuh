// qt_forward.cuh -- the forward step of the Quantization Tree algorithm
// (Algorithm III of Pages & Wilbertz, arXiv:1101.3228, Sec. 4) as one
// persistent kernel over all layers.
//
// Work item = (layer k, tile of samples).  Items are ordered layer by layer and
// handed out by an atomic counter, so uneven grid sizes N_k balance by
// themselves (the paper runs one block per layer; Sec. 4, remark after
// Algorithm III).  On a layer switch a CTA stages Gamma_k and Gamma_{k+1} into
// shared memory with bulk TMA copies (cp.async.bulk + mbarrier), which is the
// GB300 form of the paper's "grids in shared memory" design.
//
// Per sample: draw (X_k, eps_k) (qt_sampler.cuh), search the nearest cell of
// X_k in Gamma_k and of Y = A_k X_k + b_k + T_k eps_k in Gamma_{k+1} (Sec. 3.2,
// brute force as the paper chose), then add 1 to p^k_ij (Sec. 3.3: atomics;
// here a shared-memory private histogram or red.global.add into L2).
//
// Search forms:
//  * plain FP64: the exact distance D64 of the library contract, strict '<'
//    over ascending indices (ties to the lowest index);
//  * FP32 screen: scores s_j = |c_j - mu|^2 - 2 (x - mu).(c_j - mu) with FMA
//    chains on centred FP32 copies; the running minimum is tracked per chunk of
//    kChunk candidates (one 3-input min per candidate pair), the best chunk is
//    re-scored at the end for the index and the second-best score.  With
//    E(r) = (d+2) 2^-24 (r^2 + 2|x^| r) the bound on |s~_j - s_j| for a grid
//    point at distance r from the centre, a sample is certified when
//    s_2nd - s_best > E(rho) + E(r_best) + eta, rho the largest radius at which
//    a point can still beat the best (see screen_certified for the test as
//    evaluated, with its slack factors; x^ is the centred sample and eta covers
//    the FP64 rounding of the exact distance).  Uncertified samples go to the
//    exact window search of the whole warp (warp_window_nn).
#pragma once
#include <cstdint>
#include <cfloat>

#include "qt_internal.h"
#include "qt_sampler.cuh"

namespace qt {

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared, completion counted on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// One wait on the phase `parity` of an mbarrier: the thread may be suspended
// in hardware until the phase completes, for at most about 20 microseconds
// (the suspend-time hint), so waiting warps take few issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up once `budget_us` microseconds of the global timer have
// passed; budget_us < 0 gives up without waiting.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long budget_us)
{
    if (budget_us < 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    const unsigned long long lim = (unsigned long long)budget_us * 1000ull;
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > lim) return false;
    }
}

// Bound of the waits that drain a CTA's own copies before it leaves (after a
// timeout elsewhere): 20 s.
constexpr long long kDrainUs = 20000000;

__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ void record_error(DevStatus* st, int code, int where)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

__device__ __forceinline__ void count_add(void* counts, int u32, long long e, uint32_t v)
{
    if (u32) {
        asm volatile("red.global.add.u32 [%0], %1;" ::"l"((uint32_t*)counts + e), "r"(v) : "memory");
    } else {
        asm volatile("red.global.add.u64 [%0], %1;" ::"l"((unsigned long long*)counts + e),
                     "l"((unsigned long long)v)
                     : "memory");
    }
}

// Exact distance of the library contract: sum_l (z_l - x_l)^2, left to right,
// binary64, round to nearest, no contraction.
template <int DM>
__device__ __forceinline__ double dist64(const double (&z)[DM], const double* __restrict__ x, int d)
{
    double acc = 0.0;
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        if (l < d) {
            const double t = __dsub_rn(z[l], x[l]);
            acc = __dadd_rn(acc, __dmul_rn(t, t));
        }
    }
    return acc;
}

// Records of the FP32 screen: [cc, c_0 .. c_{DM-1}, 0 ...] rounded up to float4.
template <int DM>
struct Rec32 {
    static constexpr int kVec = (DM + 1 + 3) / 4;
    static constexpr int kFloats = 4 * kVec;
};
template <int DM>
struct Rec64 {
    static constexpr int kDoubles = (DM + 1) / 2 * 2;
};

// ------------------------------------------------------------------ sample access

// Exact sample (X or Y) of sample m as FP64 (regenerated for rechecks and dumps).
template <int DM>
__device__ __noinline__ void exact_sample(const ForwardParams& p, const float* spf, const double* spd, int k,
                                             unsigned long long m, bool wantY, double (&z)[DM])
{
    if (p.source == kArrays) {
        const double* src = wantY ? p.srcY : p.srcX;
#pragma unroll
        for (int l = 0; l < DM; ++l) z[l] = (l < p.d) ? src[m * (unsigned long long)p.d + l] : 0.0;
        return;
    }
    if (p.prec == 1) {
        float X[DM], Y[DM];
        pair_f32<DM>(spf, p.d, p.seed, k, m, X, Y);
#pragma unroll
        for (int l = 0; l < DM; ++l) z[l] = (double)(wantY ? Y[l] : X[l]);
    } else {
        double X[DM], Y[DM];
        pair_f64<DM>(spd, p.d, p.seed, k, m, X, Y);
#pragma unroll
        for (int l = 0; l < DM; ++l) z[l] = wantY ? Y[l] : X[l];
    }
}

// ------------------------------------------------------------------ FP32 screen

template <int DM>
struct Centred {
    float xa[DM], yb[DM];  // -2 (X - mu_A), -2 (Y - mu_B) in FP32
    float Aa, Ab;          // |X - mu_A|, |Y - mu_B| of the rounded centred values
};

// Draw (or load) sample m and centre it on the two grids (inlined form, for
// kernels that draw one sample per thread).
template <int DM>
__device__ __forceinline__ Centred<DM> centred_sample_inl(const ForwardParams& p, const float* spf, const double* spd,
                                                          const float* muA, const float* muB, int k,
                                                          unsigned long long m)
{
    Centred<DM> c;
    const int d = p.d;
    float na = 0.f, nb = 0.f;
    if (p.source == kSampler && p.prec == 1) {
        float X[DM], Y[DM];
        pair_f32<DM>(spf, d, p.seed, k, m, X, Y);
#pragma unroll
        for (int l = 0; l < DM; ++l) {
            const float ax = __fsub_rn(X[l], muA[l]);
            const float by = __fsub_rn(Y[l], muB[l]);
            na = __fmaf_rn(ax, ax, na);
            nb = __fmaf_rn(by, by, nb);
            c.xa[l] = -2.0f * ax;
            c.yb[l] = -2.0f * by;
        }
    } else {
        double X[DM], Y[DM];
        if (p.source == kSampler) {
            pair_f64<DM>(spd, d, p.seed, k, m, X, Y);
        } else {
#pragma unroll
            for (int l = 0; l < DM; ++l) {
                X[l] = (l < d) ? p.srcX[m * (unsigned long long)d + l] : 0.0;
                Y[l] = (l < d) ? p.srcY[m * (unsigned long long)d + l] : 0.0;
            }
        }
#pragma unroll
        for (int l = 0; l < DM; ++l) {
            const float ax = __double2float_rn(__dsub_rn(X[l], (double)muA[l]));
            const float by = __double2float_rn(__dsub_rn(Y[l], (double)muB[l]));
            na = __fmaf_rn(ax, ax, na);
            nb = __fmaf_rn(by, by, nb);
            c.xa[l] = -2.0f * ax;
            c.yb[l] = -2.0f * by;
        }
    }
    c.Aa = __fsqrt_rn(na);
    c.Ab = __fsqrt_rn(nb);
    return c;
}

// Out-of-line form, for kernels that draw several samples per thread.
template <int DM>
__device__ __noinline__ Centred<DM> centred_sample(const ForwardParams& p, const float* spf, const double* spd,
                                                   const float* muA, const float* muB, int k, unsigned long long m)
{
    return centred_sample_inl<DM>(p, spf, spd, muA, muB, k, m);
}

// Exact FP64 pair for the plain form.
template <int DM>
struct Exact {
    double X[DM], Y[DM];
};

template <int DM>
__device__ __noinline__ Exact<DM> exact_pair(const ForwardParams& p, const float* spf, const double* spd, int k,
                                             unsigned long long m)
{
    Exact<DM> e;
    const int d = p.d;
    if (p.source == kArrays) {
#pragma unroll
        for (int l = 0; l < DM; ++l) {
            e.X[l] = (l < d) ? p.srcX[m * (unsigned long long)d + l] : 0.0;
            e.Y[l] = (l < d) ? p.srcY[m * (unsigned long long)d + l] : 0.0;
        }
    } else if (p.prec == 1) {
        float Xf[DM], Yf[DM];
        pair_f32<DM>(spf, d, p.seed, k, m, Xf, Yf);
#pragma unroll
        for (int l = 0; l < DM; ++l) {
            e.X[l] = (double)Xf[l];
            e.Y[l] = (double)Yf[l];
        }
    } else {
        pair_f64<DM>(spd, d, p.seed, k, m, e.X, e.Y);
    }
    return e;
}

// Running minimum of the FP32 screen over one grid, per sample.
template <int S>
struct ScanState {
    float B1[S];   // best score
    float B2[S];   // smallest chunk minimum outside the best chunk
    int bc[S];     // best chunk (global chunk index)
};

template <int S>
__device__ __forceinline__ void scan_init(ScanState<S>& st)
{
#pragma unroll
    for (int s = 0; s < S; ++s) {
        st.B1[s] = __int_as_float(0x7F800000);
        st.B2[s] = __int_as_float(0x7F800000);
        st.bc[s] = 0;
    }
}

// Resolution of the best chunk, kept across segments in the streamed mode.
template <int S>
struct ResolveState {
    float S1[S];   // smallest other score inside the best chunk
    float r1[S];   // |g^| of the best record
    int rc[S];     // chunk for which idx, S1, r1 hold (-1: none)
    int idx[S];    // best record index
};

template <int S>
__device__ __forceinline__ void resolve_init(ResolveState<S>& rs)
{
#pragma unroll
    for (int s = 0; s < S; ++s) {
        rs.S1[s] = __int_as_float(0x7F800000);
        rs.r1[s] = 0.0f;
        rs.rc[s] = -1;
        rs.idx[s] = -1;
    }
}

// Re-score local chunk lc of `recs` (global chunk gc) for one sample: lowest
// index achieving B1, smallest other score of the chunk, norm of the best
// record.  Chunks are 16 records apart, which puts record q of every chunk in
// the same shared-memory banks; lane t therefore starts at record t mod 16 and
// wraps around, so that lanes whose best chunks differ read different banks
// (one vector load per 16 bytes of a record).  The outcome does not depend on
// the order: the lowest index whose score equals B1, and as the other score the
// smallest score of the rest (B1 itself when two records reach it).
template <int DM>
__device__ __forceinline__ void resolve_chunk(const float* __restrict__ recs, int lc, int gc, const float (&x)[DM],
                                              float B1, int& idx, float& S1, float& r1)
{
    constexpr int F = Rec32<DM>::kFloats;
    constexpr int V = F / 4;
    const int rot = (int)(threadIdx.x & (kChunk - 1));
    const float4* base = reinterpret_cast<const float4*>(recs) + (long long)lc * kChunk * V;
    auto load = [&](int q, float (&f)[F]) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float4 a = base[q * V + v];
            f[4 * v] = a.x;
            f[4 * v + 1] = a.y;
            f[4 * v + 2] = a.z;
            f[4 * v + 3] = a.w;
        }
    };
    int lo = kChunk, matches = 0;
    float other = __int_as_float(0x7F800000);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
        const int q = (u + rot) & (kChunk - 1);
        float f[F];
        load(q, f);
        float sc = f[0];
#pragma unroll
        for (int l = 0; l < DM; ++l) sc = __fmaf_rn(x[l], f[1 + l], sc);
        if (sc == B1) {
            ++matches;
            lo = min(lo, q);
        } else {
            other = fminf(other, sc);
        }
    }
    S1 = matches >= 2 ? fminf(other, B1) : other;
    idx = -1;
    r1 = 0.0f;
    if (lo < kChunk) {
        idx = gc * kChunk + lo;
        float f[F];
        load(lo, f);
        float n2 = 0.0f;
#pragma unroll
        for (int l = 0; l < DM; ++l) n2 = __fmaf_rn(f[1 + l], f[1 + l], n2);
        r1 = __fsqrt_rn(n2);
    }
}

template <int DM>
__device__ __forceinline__ void resolve_one(const float* __restrict__ recs, int bc, const float (&x)[DM], float B1,
                                            int& idx, float& S1, float& r1)
{
    resolve_chunk<DM>(recs, bc, bc, x, B1, idx, S1, r1);
}


// ---- packed FP32 pairs (fma.rn.f32x2: two independent FP32 FMAs, each rounded
// to nearest, so each lane's result is bit-identical to the scalar FMA)
__device__ __forceinline__ uint64_t pack2(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t x, uint64_t c, uint64_t a)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(c), "l"(a));
    return r;
}
template <int V>
__device__ __forceinline__ void load_pair(const float4* __restrict__ r4, int j, float4 (&a)[V], float4 (&b)[V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        a[v] = r4[j * V + v];
        b[v] = r4[(j + 1) * V + v];
    }
}

// Scan `nchunk` chunks of records (global chunk index of the first: c0) for S
// centred, scaled samples xs = -2 x^.  The next pair of records is loaded
// while the current pair is scored.
template <int DM, int S>
__device__ __forceinline__ void screen_scan(const float* __restrict__ recs, int nchunk, int c0,
                                            const float (&xs)[S][DM], ScanState<S>& st)
{
    constexpr int V = Rec32<DM>::kVec;
    const float4* r4 = reinterpret_cast<const float4*>(recs);
    const int last = nchunk * kChunk - 2;
    // samples 2p and 2p + 1 share one packed FMA per record element: their
    // coordinates side by side, the record's element broadcast to both lanes
    uint64_t xp[S / 2 > 0 ? S / 2 : 1][DM];
#pragma unroll
    for (int sp = 0; sp < S / 2; ++sp)
#pragma unroll
        for (int l = 0; l < DM; ++l) xp[sp][l] = pack2(xs[2 * sp][l], xs[2 * sp + 1][l]);
    float4 na[V], nb[V];
    load_pair<V>(r4, 0, na, nb);
    for (int c = 0; c < nchunk; ++c) {
        float mc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) mc[s] = __int_as_float(0x7F800000);
#pragma unroll
        for (int q = 0; q < kChunk; q += 2) {
            float4 ca[V], cb[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                ca[v] = na[v];
                cb[v] = nb[v];
            }
            const int jn = min(c * kChunk + q + 2, last);
            load_pair<V>(r4, jn, na, nb);
            const float* ra = reinterpret_cast<const float*>(ca);
            const float* rb = reinterpret_cast<const float*>(cb);
            if constexpr (S >= 2) {
                uint64_t ea[DM + 1], eb[DM + 1];
#pragma unroll
                for (int e = 0; e <= DM; ++e) {
                    ea[e] = pack2(ra[e], ra[e]);
                    eb[e] = pack2(rb[e], rb[e]);
                }
#pragma unroll
                for (int sp = 0; sp < S / 2; ++sp) {
                    uint64_t aa = ea[0], bb = eb[0];
#pragma unroll
                    for (int l = 0; l < DM; ++l) {
                        aa = ffma2(xp[sp][l], ea[1 + l], aa);
                        bb = ffma2(xp[sp][l], eb[1 + l], bb);
                    }
                    float a0, a1, b0, b1;
                    unpack2(aa, a0, a1);
                    unpack2(bb, b0, b1);
                    mc[2 * sp] = min3f(mc[2 * sp], a0, b0);
                    mc[2 * sp + 1] = min3f(mc[2 * sp + 1], a1, b1);
                }
            }
#pragma unroll
            for (int s = (S / 2) * 2; s < S; ++s) {
                float sa = ra[0], sb = rb[0];
#pragma unroll
                for (int l = 0; l < DM; ++l) {
                    sa = __fmaf_rn(xs[s][l], ra[1 + l], sa);
                    sb = __fmaf_rn(xs[s][l], rb[1 + l], sb);
                }
                mc[s] = min3f(mc[s], sa, sb);
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            st.B2[s] = fminf(st.B2[s], fmaxf(mc[s], st.B1[s]));
            const bool nw = mc[s] < st.B1[s];
            st.B1[s] = fminf(st.B1[s], mc[s]);
            st.bc[s] = nw ? c0 + c : st.bc[s];
        }
    }
}

// Streamed mode: for samples whose best chunk lies in the scanned records
// [c0, c0 + nchunk) and is not resolved yet, resolve it while it is in
// shared memory.
template <int DM, int S>
__device__ __forceinline__ void screen_resolve(const float* __restrict__ recs, int nchunk, int c0,
                                               const float (&xs)[S][DM], const ScanState<S>& st,
                                               ResolveState<S>& rs)
{
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int lc = st.bc[s] - c0;
        if (st.bc[s] == rs.rc[s] || lc < 0 || lc >= nchunk) continue;
        resolve_chunk<DM>(recs, lc, st.bc[s], xs[s], st.B1[s], rs.idx[s], rs.S1[s], rs.r1[s]);
        rs.rc[s] = st.bc[s];
    }
}

// Certificate of the screened argmin (exact reasoning in the design notes):
// with a = x - mu, g_j = c_j - mu, s_j = |g_j|^2 - 2 a.g_j the exact score and
// s~_j the FP32 score, |s~_j - s_j| <= E(|g_j|), E(r) = (d+2) 2^-24 (r^2 + 2|a| r).
// Every j with |g_j| > rho = |a| + sqrt(|a|^2 + s~_best + E(r_best)) has
// s_j > s_best, and every other j has s_j >= s~_2nd - E(rho); so the screened
// best is the exact FP64 argmin when s~_2nd - s~_best > E(rho) + E(r_best) + eta
// (eta covers the FP64 rounding of the exact distance).  Slack factors absorb
// the FP32 evaluation of this test.
__device__ __forceinline__ bool screen_certified(int d, float A, float B1, float second, float r1n)
{
    const float Ap = A * (1.0f + 0x1p-18f);
    const float cd = (float)(d + 2) * 0x1p-24f * (1.0f + 0x1p-10f);
    const float r1 = r1n * (1.0f + 0x1p-18f);
    const float E1 = cd * (r1 * r1 + 2.0f * Ap * r1);
    const float U = B1 + E1;
    const float A2 = Ap * Ap;
    const float eta = 0x1p-44f * (A2 + fabsf(B1) + E1);
    const float rad = fmaxf(A2 + U + 0x1p-18f * (A2 + fabsf(U)) + eta, 0.0f);
    const float rho = Ap + __fsqrt_rn(rad);
    const float Erho = cd * (rho * rho + 2.0f * Ap * rho);
    const float thr = (Erho + E1 + eta) * (1.0f + 0x1p-16f);
    return (second - B1) > thr;
}

// Exact window search for one lane's sample (broadcast from lane `src`): the
// warp screens the whole grid in FP32, then evaluates the exact FP64 distance
// only on the records whose FP32 score lies inside the window the certificate's
// bounds allow, and returns the lowest index among the smallest distances.
template <int DM>
__device__ __noinline__ int warp_window_nn(const float (&xs)[DM], float A, const double (&z)[DM], int src,
                                           const float* __restrict__ recs, int Npad, const double* __restrict__ g64,
                                           int N, int d)
{
    constexpr int F = Rec32<DM>::kFloats;
    float x[DM];
    double zz[DM];
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        x[l] = __shfl_sync(0xFFFFFFFFu, xs[l], src);
        zz[l] = __shfl_sync(0xFFFFFFFFu, z[l], src);
    }
    const float Av = __shfl_sync(0xFFFFFFFFu, A, src);
    const int lane = threadIdx.x & 31;
    // a lane scores records j, j + 32, j + 64, j + 96 (loads in flight together),
    // then takes them in increasing index order
    constexpr int kU = 4;
    auto score = [&](int j) {
        const float4* r4 = reinterpret_cast<const float4*>(recs + (long long)j * F);
        float f[F];
#pragma unroll
        for (int v = 0; v < F / 4; ++v) {
            const float4 a = r4[v];
            f[4 * v] = a.x;
            f[4 * v + 1] = a.y;
            f[4 * v + 2] = a.z;
            f[4 * v + 3] = a.w;
        }
        float sc = f[0];
#pragma unroll
        for (int l = 0; l < DM; ++l) sc = __fmaf_rn(x[l], f[1 + l], sc);
        return sc;
    };
    float b1 = __int_as_float(0x7F800000);
    int i1 = 0x7FFFFFFF;
    for (int j0 = lane; j0 < N; j0 += 32 * kU) {
        float sc[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) sc[u] = score(min(j0 + 32 * u, N - 1));
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (j0 + 32 * u < N && sc[u] < b1) {
                b1 = sc[u];
                i1 = j0 + 32 * u;
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const float ob = __shfl_xor_sync(0xFFFFFFFFu, b1, off);
        const int oi = __shfl_xor_sync(0xFFFFFFFFu, i1, off);
        if (ob < b1 || (ob == b1 && oi < i1)) {
            b1 = ob;
            i1 = oi;
        }
    }
    // window bound (same bounds as the certificate, with slack)
    const float* r = recs + (long long)i1 * F;
    float n2 = 0.0f;
#pragma unroll
    for (int l = 0; l < DM; ++l) n2 = __fmaf_rn(r[1 + l], r[1 + l], n2);
    const float Ap = Av * (1.0f + 0x1p-18f);
    const float cd = (float)(d + 2) * 0x1p-24f * (1.0f + 0x1p-10f);
    const float r1 = __fsqrt_rn(n2) * (1.0f + 0x1p-18f);
    const float E1 = cd * (r1 * r1 + 2.0f * Ap * r1);
    const float U = b1 + E1;
    const float A2 = Ap * Ap;
    const float eta = 0x1p-44f * (A2 + fabsf(b1) + E1);
    const float rad = fmaxf(A2 + U + 0x1p-18f * (A2 + fabsf(U)) + eta, 0.0f);
    const float rho = Ap + __fsqrt_rn(rad);
    const float Erho = cd * (rho * rho + 2.0f * Ap * rho);
    const float lim = b1 + (E1 + Erho + eta) * 1.25f + 0x1p-20f * fabsf(b1) + 0x1p-100f;
    // exact distances on the window only
    double best = __longlong_as_double(0x7FF0000000000000LL);
    int bi = 0x7FFFFFFF;
    for (int j0 = lane; j0 < N; j0 += 32 * kU) {
        float sc[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) sc[u] = score(min(j0 + 32 * u, N - 1));
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int j = j0 + 32 * u;
            if (j < N && sc[u] <= lim) {
                const double dj = dist64<DM>(zz, g64 + (long long)j * d, d);
                if (dj < best) {
                    best = dj;
                    bi = j;
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const double ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
        const int oi = __shfl_xor_sync(0xFFFFFFFFu, bi, off);
        if (ob < best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    (void)Npad;
    return bi;
}

// ------------------------------------------------------------------ the kernel

// Small dimension classes keep two CTAs (16 warps) resident per SM.
template <int DM, int S, int FORM, bool STREAMED>
__global__ void __launch_bounds__(256, (DM <= 4 ? 2 : 1)) forward_kernel(const ForwardParams p)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ long long s_item;
    __shared__ LayerDesc s_L;
    __shared__ GridInfo s_GA, s_GB;
    __shared__ __align__(16) float s_pf[param_count(DM)];
    __shared__ __align__(16) double s_pd[param_count(DM)];
    __shared__ int s_abort;
    __shared__ __align__(8) unsigned long long s_ring_bar[kSlots];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int d = p.d;
    const uint32_t bar = smem_u32(&s_bar);
    unsigned char* grid_sm = dsm;
    uint32_t* hist = reinterpret_cast<uint32_t*>(dsm + p.smem_grid_bytes);

    if (tid == 0) {
        mbar_init(bar, 1);
        for (int t = 0; t < kSlots; ++t) mbar_init(smem_u32(&s_ring_bar[t]), 1);
        fence_proxy_async();
        s_abort = 0;
    }
    __syncthreads();

    int cur = -1;
    uint32_t phase = 0;
    uint32_t ring_phase[kSlots];
#pragma unroll
    for (int t = 0; t < kSlots; ++t) ring_phase[t] = 0;
    bool hist_live = false;

    while (true) {
        if (tid == 0) {
            long long it = -1;
            if (*((volatile int32_t*)&p.status->code) == 0)
                it = (long long)atomicAdd(&p.status->queue, 1ull);
            s_item = it;
        }
        __syncthreads();
        const long long item = s_item;
        if (item < 0 || item >= p.total_items) break;

        // ---- locate the layer of this item (items are grouped layer by layer)
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
            // ---- flush the private histogram of the previous layer
            if (hist_live) {
                const int ent = s_L.NA * s_L.NB;
                for (int e = tid; e < ent; e += blockDim.x) {
                    const uint32_t v = hist[e];
                    if (v) {
                        count_add(p.counts, p.counts_u32, s_L.coff + e, v);
                        hist[e] = 0;
                    }
                }
                hist_live = false;
            }
            __syncthreads();
            if (tid == 0) {
                s_L = p.layers[k];
                s_GA = p.grids[s_L.gridA];
                s_GB = p.grids[s_L.gridB];
            }
            __syncthreads();
            // ---- stage both grids with bulk copies (TMA engine); the streamed
            // mode stages segments per tile instead
            const bool resident = !STREAMED;
            if (tid == 0 && resident) {
                uint32_t bytesA, bytesB;
                const void *srcA, *srcB;
                if (FORM == kF32Recheck) {
                    bytesA = (uint32_t)s_L.NApad * Rec32<DM>::kFloats * 4u;
                    bytesB = (uint32_t)s_L.NBpad * Rec32<DM>::kFloats * 4u;
                    srcA = p.rec32 + s_L.roffA * Rec32<DM>::kFloats;
                    srcB = p.rec32 + s_L.roffB * Rec32<DM>::kFloats;
                } else {
                    bytesA = (uint32_t)s_L.NApad * Rec64<DM>::kDoubles * 8u;
                    bytesB = (uint32_t)s_L.NBpad * Rec64<DM>::kDoubles * 8u;
                    srcA = p.rec64 + s_L.roffA * Rec64<DM>::kDoubles;
                    srcB = p.rec64 + s_L.roffB * Rec64<DM>::kDoubles;
                }
                fence_proxy_async();
                mbar_arrive_expect_tx(bar, bytesA + bytesB);
                bulk_g2s(smem_u32(grid_sm), srcA, bytesA, bar);
                bulk_g2s(smem_u32(grid_sm + bytesA), srcB, bytesB, bar);
            }
            // ---- sampler parameters and private histogram
            if (p.source == kSampler) {
                const int pc = param_count(d);
                for (int e = tid; e < pc; e += blockDim.x) {
                    s_pf[e] = p.params_f[(long long)k * p.params_stride + e];
                    s_pd[e] = p.params_d[(long long)k * p.params_stride + e];
                }
            }
            if (s_L.hist_smem) {
                const int ent = s_L.NA * s_L.NB;
                for (int e = tid; e < ent; e += blockDim.x) hist[e] = 0;
                hist_live = true;
            }
            // ---- wait for the grids (bounded)
            const bool ok = !resident || mbar_wait_bounded(bar, phase, p.spin_budget);
            if (!ok) {
                // give up: record the timeout, let the copies land (bounded, fixed
                // budget), then leave the kernel without touching the results
                if (tid == 0) {
                    record_error(p.status, 4 /* QT_ETIMEOUT */, 1);
                    s_abort = 1;
                }
                mbar_wait_bounded(bar, phase, kDrainUs);
            }
            if (resident) phase ^= 1u;
            __syncthreads();
            if (s_abort) break;
            cur = k;
        }

        const LayerDesc& L = s_L;
        const unsigned long long mtile = (unsigned long long)(item - L.item_begin) * (unsigned long long)p.tile;
        unsigned long long ms[S];
        bool valid[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            ms[s] = mtile + (unsigned long long)(s * blockDim.x + tid);
            valid[s] = ms[s] < p.M;
        }

        int ci[S], cj[S];

        if (FORM == kF32Recheck) {
            // ---- centred, scaled FP32 copies of X (grid A) and Y (grid B)
            float xa[S][DM], yb[S][DM];
            float Aa[S], Ab[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const unsigned long long m = valid[s] ? ms[s] : mtile;
                const Centred<DM> c = centred_sample<DM>(p, s_pf, s_pd, s_GA.mu, s_GB.mu, k, m);
#pragma unroll
                for (int l = 0; l < DM; ++l) {
                    xa[s][l] = c.xa[l];
                    yb[s][l] = c.yb[l];
                }
                Aa[s] = c.Aa;
                Ab[s] = c.Ab;
            }
            bool needA[S], needB[S];
            if constexpr (!STREAMED) {
                // ---- resident mode: both grids staged in shared memory at the layer switch
                const float* recA = reinterpret_cast<const float*>(grid_sm);
                const float* recB = recA + (long long)L.NApad * Rec32<DM>::kFloats;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const float* rec = g == 0 ? recA : recB;
                    const int nch = (g == 0 ? L.NApad : L.NBpad) / kChunk;
                    ScanState<S> st;
                    scan_init<S>(st);
                    if (g == 0) screen_scan<DM, S>(rec, nch, 0, xa, st);
                    else screen_scan<DM, S>(rec, nch, 0, yb, st);
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        int idx;
                        float S1, r1;
                        if (g == 0) resolve_one<DM>(rec, st.bc[s], xa[s], st.B1[s], idx, S1, r1);
                        else resolve_one<DM>(rec, st.bc[s], yb[s], st.B1[s], idx, S1, r1);
                        const float second = fminf(st.B2[s], S1);
                        const bool cert =
                            idx >= 0 && screen_certified(d, g == 0 ? Aa[s] : Ab[s], st.B1[s], second, r1);
                        if (g == 0) {
                            ci[s] = idx;
                            needA[s] = !cert && valid[s];
                        } else {
                            cj[s] = idx;
                            needB[s] = !cert && valid[s];
                        }
                    }
                }
            } else {
                // ---- streamed mode: segments of kSeg records through a two-slot
                // ring of bulk copies; the CTA walks the segments in lockstep
                const int seg_recs = p.seg_records;
                const uint32_t seg_bytes = (uint32_t)seg_recs * Rec32<DM>::kFloats * 4u;
                const int nA = L.segA, nB = L.segB, ntot = nA + nB;
                auto seg_src = [&](int t, uint32_t& bytes) -> const float* {
                    const bool isA = t < nA;
                    const int ts = isA ? t : t - nA;
                    const int npad = isA ? L.NApad : L.NBpad;
                    const int first = ts * seg_recs;
                    const int cnt = min(seg_recs, npad - first);
                    bytes = (uint32_t)cnt * Rec32<DM>::kFloats * 4u;
                    return p.rec32 + ((isA ? L.roffA : L.roffB) + first) * Rec32<DM>::kFloats;
                };
                bool pending[kSlots];   // a copy is in flight on this slot
#pragma unroll
                for (int t = 0; t < kSlots; ++t) pending[t] = t < ntot;
                if (tid == 0) {
                    fence_proxy_async();
#pragma unroll
                    for (int t = 0; t < kSlots; ++t) {
                        if (t < ntot) {
                            uint32_t bytes;
                            const float* src = seg_src(t, bytes);
                            const uint32_t sb = smem_u32(&s_ring_bar[t]);
                            mbar_arrive_expect_tx(sb, bytes);
                            bulk_g2s(smem_u32(grid_sm + t * seg_bytes), src, bytes, sb);
                        }
                    }
                }
                ScanState<S> st;
                ResolveState<S> rs;
                scan_init<S>(st);
                resolve_init<S>(rs);
                for (int t = 0; t < ntot; ++t) {
                    const int slot = t % kSlots;
                    const bool ok = mbar_wait_bounded(smem_u32(&s_ring_bar[slot]), ring_phase[slot], p.spin_budget);
                    if (!ok && tid == 0) {
                        record_error(p.status, 4 /* QT_ETIMEOUT */, 3);
                        s_abort = 1;
                    }
                    if (!ok) mbar_wait_bounded(smem_u32(&s_ring_bar[slot]), ring_phase[slot], kDrainUs);
                    ring_phase[slot] ^= 1u;
                    pending[slot] = false;
                    const bool isA = t < nA;
                    const int ts = isA ? t : t - nA;
                    const int npad = isA ? L.NApad : L.NBpad;
                    const int cnt = min(seg_recs, npad - ts * seg_recs);
                    const float* rec = reinterpret_cast<const float*>(grid_sm + slot * seg_bytes);
                    const int c0 = ts * seg_recs / kChunk;
                    if (isA) {
                        screen_scan<DM, S>(rec, cnt / kChunk, c0, xa, st);
                        screen_resolve<DM, S>(rec, cnt / kChunk, c0, xa, st, rs);
                    } else {
                        screen_scan<DM, S>(rec, cnt / kChunk, c0, yb, st);
                        screen_resolve<DM, S>(rec, cnt / kChunk, c0, yb, st, rs);
                    }
                    if (t == nA - 1 || t == ntot - 1) {
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            const float second = fminf(st.B2[s], rs.S1[s]);
                            const bool cert = rs.idx[s] >= 0 &&
                                              screen_certified(d, isA ? Aa[s] : Ab[s], st.B1[s], second, rs.r1[s]);
                            if (isA) {
                                ci[s] = rs.idx[s];
                                needA[s] = !cert && valid[s];
                            } else {
                                cj[s] = rs.idx[s];
                                needB[s] = !cert && valid[s];
                            }
                        }
                        scan_init<S>(st);
                        resolve_init<S>(rs);
                    }
                    __syncthreads();   // every warp is done with this slot
                    if (s_abort) break;
                    if (t + kSlots < ntot) {
                        pending[slot] = true;
                        if (tid == 0) {
                            uint32_t bytes;
                            const float* src = seg_src(t + kSlots, bytes);
                            const uint32_t sb = smem_u32(&s_ring_bar[slot]);
                            fence_proxy_async();
                            mbar_arrive_expect_tx(sb, bytes);
                            bulk_g2s(smem_u32(grid_sm + slot * seg_bytes), src, bytes, sb);
                        }
                    }
                }
                if (s_abort) {
                    // let the copies still in flight land before the CTA leaves
#pragma unroll
                    for (int t = 0; t < kSlots; ++t)
                        if (pending[t]) mbar_wait_bounded(smem_u32(&s_ring_bar[t]), ring_phase[t], kDrainUs);
                    break;
                }
            }
            // ---- exact FP64 recheck of uncertified searches, one warp per search
#pragma unroll
            for (int s = 0; s < S; ++s) {
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const bool need = g == 0 ? needA[s] : needB[s];
                    unsigned mask = __ballot_sync(0xFFFFFFFFu, need);
                    if (mask == 0) continue;
                    double z[DM];
                    if (need) exact_sample<DM>(p, s_pf, s_pd, k, ms[s], g == 1, z);
                    const GridInfo& G = g == 0 ? s_GA : s_GB;
                    const double* g64 = p.g64 + G.goff * d;
                    const int N = g == 0 ? L.NA : L.NB;
                    float xsv[DM];
#pragma unroll
                    for (int l = 0; l < DM; ++l) xsv[l] = g == 0 ? xa[s][l] : yb[s][l];
                    const float Av = g == 0 ? Aa[s] : Ab[s];
                    while (mask) {
                        const int src = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const int r = warp_window_nn<DM>(xsv, Av, z, src, p.rec32 + G.roff * Rec32<DM>::kFloats,
                                                         G.Npad, g64, N, d);
                        if (lane == src) {
                            if (g == 0) ci[s] = r; else cj[s] = r;
                        }
                        if (lane == 0) atomicAdd(&p.status->rechecks, 1ull);
                    }
                }
            }
        } else {
            // ---- plain FP64 brute force (exact by construction)
            constexpr int R64 = Rec64<DM>::kDoubles;
            const double* recA = reinterpret_cast<const double*>(grid_sm);
            const double* recB = recA + (long long)L.NApad * R64;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const unsigned long long m = valid[s] ? ms[s] : mtile;
                const Exact<DM> ex = exact_pair<DM>(p, s_pf, s_pd, k, m);
                const double(&X)[DM] = ex.X;
                const double(&Y)[DM] = ex.Y;
                double bx = dist64<DM>(X, recA, d), by = dist64<DM>(Y, recB, d);
                int ix = 0, iy = 0;
                for (int j = 1; j < L.NA; ++j) {
                    const double dj = dist64<DM>(X, recA + (long long)j * R64, d);
                    if (dj < bx) {
                        bx = dj;
                        ix = j;
                    }
                }
                for (int j = 1; j < L.NB; ++j) {
                    const double dj = dist64<DM>(Y, recB + (long long)j * R64, d);
                    if (dj < by) {
                        by = dj;
                        iy = j;
                    }
                }
                ci[s] = ix;
                cj[s] = iy;
            }
        }

        // ---- counters p^k_ij (Sec. 3.3), per-sample cells, dumps
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!valid[s]) continue;
            const int i = ci[s], j = cj[s];
            if ((unsigned)i >= (unsigned)L.NA || (unsigned)j >= (unsigned)L.NB) {
                record_error(p.status, 6 /* QT_EDEVICE */, 2);
                continue;
            }
            const long long e = (long long)i * L.NB + j;
            if (L.hist_smem) atomicAdd(&hist[e], 1u);
            else count_add(p.counts, p.counts_u32, L.coff + e, 1u);
            if (p.cellsA) {
                p.cellsA[ms[s]] = i;
                p.cellsB[ms[s]] = j;
            }
            if (p.dump_count > 0 && (ms[s] % (unsigned long long)p.dump_stride) == 0ull) {
                const unsigned long long t = ms[s] / (unsigned long long)p.dump_stride;
                if (t < (unsigned long long)p.dump_count) {
                    const long long row = (long long)k * p.dump_count + (long long)t;
                    double zx[DM], zy[DM];
                    exact_sample<DM>(p, s_pf, s_pd, k, ms[s], false, zx);
                    exact_sample<DM>(p, s_pf, s_pd, k, ms[s], true, zy);
                    for (int l = 0; l < d; ++l) {
                        p.dumpX[row * d + l] = zx[l];
                        p.dumpY[row * d + l] = zy[l];
                    }
                    p.dumpI[row] = i;
                    p.dumpJ[row] = j;
                }
            }
        }
        __syncthreads();
    }

    // ---- final flush of the private histogram
    if (hist_live) {
        const int ent = s_L.NA * s_L.NB;
        for (int e = tid; e < ent; e += blockDim.x) {
            const uint32_t v = hist[e];
            if (v) count_add(p.counts, p.counts_u32, s_L.coff + e, v);
        }
    }
}

}  // namespace qt
