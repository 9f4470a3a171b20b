// qt_forward_tc.cu -- the tensor-core screen (qt_forward_tc.cuh) with its
// samples drawn by a separate pass, the preparation of the FP16 operand tiles,
// and the dispatch of both screen layouts.
#include "qt_forward_tc.cuh"

namespace qt {

// FP16 operand tiles of every grid: row j of grid g (tile j/256) holds
// [g_hi (dm), g_lo (dm), g_hi (dm), cc_hi, cc_lo, 0 ...] of sigma g^ and
// sigma^2 cc (coordinates l >= d zero); padded rows carry cc_hi = +inf.
// Layout inside a tile: core matrices of 8 rows x 8 halves, (row block,
// K block) at ((n/8)(K/8) + k/8) * 64.
__global__ void prep_tc_tiles_kernel(const float* __restrict__ rec32, GridInfo* gi, int ngrids, int d, int dm,
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
            put(dm + l, lo16);
            put(2 * dm + l, h);
        }
        const float c = sg * sg * rc[0];
        const __half ch = __float2half_rn(c);
        put(3 * dm, ch);
        put(3 * dm + 1, __float2half_rn(c - __half2float(ch)));
    } else {
        put(3 * dm, __float2half_rn(__int_as_float(0x7F800000)));
    }
}

// Draw pass of the DRAW_IN = false layout: one CTA of 128 threads per work
// item of [item_lo, item_hi); thread t draws row t (the same function the
// certifier warps use inside the screen kernel) into the item's record of
// p.tc_items.
template <int DM, int KT>
__global__ void __launch_bounds__(kTcTileM) tc_draw_kernel(const ForwardParams p)
{
    constexpr int K = 16 * KT;
    constexpr long long kItemOp = tc_item_op_bytes(K), kItemCert = tc_item_cert_bytes(DM);
    __shared__ int s_k;
    __shared__ long long s_beg;
    const int t = threadIdx.x;
    const long long item = p.item_lo + blockIdx.x;
    if (t == 0) {
        s_k = layer_of(p, item);
        s_beg = p.layers[s_k].item_begin;
    }
    __syncthreads();
    const int k = s_k;
    const unsigned long long mtile = (unsigned long long)(item - s_beg) * kTcTileM;
    const unsigned long long ms = mtile + (unsigned long long)t;
    unsigned char* dst = p.tc_items + (item - p.item_lo) * (kItemOp + kItemCert);
    draw_row<DM, K>(p, k, p.layers[k], ms < p.M ? ms : mtile, t, dst, reinterpret_cast<float*>(dst + kItemOp));
}

template <int DM, int KT>
static cudaError_t launch_draw(const ForwardParams& p, cudaStream_t st)
{
    const long long n = p.item_hi - p.item_lo;
    if (n < 1) return cudaSuccess;
    tc_draw_kernel<DM, KT><<<(unsigned)n, kTcTileM, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tc_draw(int dm, const ForwardParams& p, cudaStream_t st)
{
    if (dm == 2) return launch_draw<2, 1>(p, st);
    if (dm == 4) return launch_draw<4, 1>(p, st);
    if (dm == 6) return launch_draw<6, 2>(p, st);
    if (dm == 8) return launch_draw<8, 2>(p, st);
    if (dm == 10) return launch_draw<10, 2>(p, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tc_forward(int dm, const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st)
{
    if (p.tc_draw_in) return launch_tc_forward_drawin(dm, p, dyn, num_sms, bps, st);
    if (dm == 2) return launch_tc<2, 1, false>(p, dyn, num_sms, bps, st);
    if (dm == 4) return launch_tc<4, 1, false>(p, dyn, num_sms, bps, st);
    if (dm == 6) return launch_tc<6, 2, false>(p, dyn, num_sms, bps, st);
    if (dm == 8) return launch_tc<8, 2, false>(p, dyn, num_sms, bps, st);
    if (dm == 10) return launch_tc<10, 2, false>(p, dyn, num_sms, bps, st);
    return cudaErrorInvalidValue;
}

}  // namespace qt
