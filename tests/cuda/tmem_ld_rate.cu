// tmem_ld_rate.cu -- test program: how fast warps can read tensor memory with
// the reduction load that the tensor-core screen's epilogue uses
// (tcgen05.ld.red.32x32b.x16.min.f32, four loads per wait, 16 loads for a
// 256-column accumulator).  One CTA per SM allocates all 512 columns and fills
// them with tcgen05.st; then W warps (W = 4, 8, 16) read their lanes' share of
// one 256-column accumulator, `reps` times over, folding the chunk minima into
// a running minimum that is written out (so that no load is dead).  Prints, per
// W, the accumulator elements read per SM per clock cycle at the maximum SM
// clock, and the cycles one warp takes per 256-column accumulator.
// A second kernel times the tensor-core round trip without any read: one
// thread issues the two K = 16 MMAs of a 128 x 256 x 32 FP16 tile (the screen's
// tile at K = 32) into a 256-column accumulator, commits them to an mbarrier
// and waits for it, `reps` times; with `inflight` = 2 it keeps two
// accumulators busy, as the screen's two warpgroups do; with `group` = 2 it
// issues both accumulators' tiles before one commit.  Prints the cycles (at the
// maximum SM clock) per commit group.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CHECK(x)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess) {                                                          \
            printf("cuda error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return 1;                                                                     \
        }                                                                                 \
    } while (0)

__device__ __forceinline__ void min4(uint32_t taddr, float& m0, float& m1, float& m2, float& m3)
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

template <int W>
__global__ void __launch_bounds__(W * 32, 1) read_rate(int reps, float* out)
{
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tmem)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = s_tmem + ((uint32_t)((warp & 3) * 32) << 16);
    if (warp < 4) {
        // fill all 512 columns of this warp's lanes, 8 columns per store
        for (int c = 0; c < 512; c += 8) {
            uint32_t v[8];
            for (int u = 0; u < 8; ++u) v[u] = __float_as_uint((float)(((lane * 7 + (c + u) * 13) % 97) - 48));
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(tm + c),
                         "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                         : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warps with the same lanes alternate between the two 256-column accumulators
    const uint32_t acc = tm + (uint32_t)(((warp >> 2) & 1) * 256);
    float m = 3.0e38f;
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float a, b, c, d;
            min4(acc + (uint32_t)(q * 64), a, b, c, d);
            m = fminf(m, fminf(fminf(a, b), fminf(c, d)));
        }
    }
    out[(size_t)blockIdx.x * W * 32 + t] = m;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(512u) : "memory");
}

__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    // shared-memory matrix descriptor, canonical K-major layout, no swizzle
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded: gives up after about a second of the global timer
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity)
{
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!bar_try(bar, parity)) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) return false;
    }
    return true;
}

__global__ void __launch_bounds__(128, 1) mma_round_trip(int reps, int inflight, int group, int* fail)
{
    extern __shared__ __align__(1024) unsigned char sm[];   // A: 128 x 32 FP16 (8 KB), B: 256 x 32 FP16 (16 KB)
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5;
    for (int e = t; e < (24 * 1024) / 4; e += 128) reinterpret_cast<uint32_t*>(sm)[e] = 0u;
    if (t == 0) {
        for (int b = 0; b < 2; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&s_bar[b]))
                         : "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tmem)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(sm), b = a + 8 * 1024;
        const uint32_t idesc = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        uint32_t ph[2] = {0u, 0u};
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r) {
            const int k = inflight == 2 ? (r & 1) : 0;
            if (r >= inflight) {
                // the accumulator's previous tile is complete
                ok = bar_wait((uint32_t)__cvta_generic_to_shared(&s_bar[k]), ph[k]);
                ph[k] ^= 1u;
            }
            for (int gi = 0; gi < group; ++gi) {
            const uint32_t d = s_tmem + (uint32_t)((group > 1 ? gi : k) * 256);
            for (int s = 0; s < 2; ++s) {
                const uint64_t ad = desc(a + s * 256, 128, 32 * 16), bd = desc(b + s * 256, 128, 32 * 16);
                const uint32_t accum = s > 0 ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                    : "memory");
            }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(&s_bar[k]))
                         : "memory");
        }
        // the last tiles of both accumulators
        for (int k = 0; k < inflight && ok; ++k) ok = bar_wait((uint32_t)__cvta_generic_to_shared(&s_bar[k]), ph[k]);
        if (!ok) atomicAdd(fail, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(512u) : "memory");
}

static int run_mma(int sms, double clk_mhz, int inflight, int group)
{
    const int reps = 20000;
    int* dfail;
    CHECK(cudaMalloc(&dfail, 4));
    CHECK(cudaMemset(dfail, 0, 4));
    const int dyn = 120 * 1024;   // one CTA per SM
    CHECK(cudaFuncSetAttribute(mma_round_trip, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    mma_round_trip<<<sms, 128, dyn>>>(reps / 10, inflight, group, dfail);
    CHECK(cudaGetLastError());
    CHECK(cudaDeviceSynchronize());
    cudaEvent_t e0, e1;
    CHECK(cudaEventCreate(&e0));
    CHECK(cudaEventCreate(&e1));
    CHECK(cudaEventRecord(e0));
    mma_round_trip<<<sms, 128, dyn>>>(reps, inflight, group, dfail);
    CHECK(cudaEventRecord(e1));
    CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CHECK(cudaEventElapsedTime(&ms, e0, e1));
    int fail = 0;
    CHECK(cudaMemcpy(&fail, dfail, 4, cudaMemcpyDeviceToHost));
    const double cyc = ms * 1e-3 * clk_mhz * 1e6 / reps;
    const double flops = 2.0 * 128 * 256 * 32 * group * reps * sms / (ms * 1e-3) / 1e12;
    printf("tmem_ld_rate mma_tile inflight %d group %d cycles_per_group %.0f tflops %.1f timeouts %d\n", inflight, group,
           cyc, flops, fail);
    CHECK(cudaFree(dfail));
    return fail ? 1 : 0;
}

template <int W>
static int run(int sms, double clk_mhz, float* dout)
{
    const int reps = 20000;
    cudaEvent_t e0, e1;
    CHECK(cudaEventCreate(&e0));
    CHECK(cudaEventCreate(&e1));
    // one CTA per SM: each takes more than half of the SM's shared memory
    const int dyn = 120 * 1024;
    CHECK(cudaFuncSetAttribute(read_rate<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    read_rate<W><<<sms, W * 32, dyn>>>(reps / 10, dout);   // warm-up
    CHECK(cudaGetLastError());
    CHECK(cudaDeviceSynchronize());
    CHECK(cudaEventRecord(e0));
    read_rate<W><<<sms, W * 32, dyn>>>(reps, dout);
    CHECK(cudaEventRecord(e1));
    CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CHECK(cudaEventElapsedTime(&ms, e0, e1));
    // elements read: every thread reads 256 columns per repetition
    const double elems = (double)sms * W * 32 * 256.0 * reps;
    const double per_sm_cycle = elems / sms / (ms * 1e-3 * clk_mhz * 1e6);
    const double warp_cycles = ms * 1e-3 * clk_mhz * 1e6 / reps;   // one warp, one 256-column accumulator
    printf("tmem_ld_rate warps %d elems_per_sm_cycle %.2f warp_cycles_per_acc %.0f ms %.3f\n", W, per_sm_cycle,
           warp_cycles, ms);
    CHECK(cudaEventDestroy(e0));
    CHECK(cudaEventDestroy(e1));
    return 0;
}

int main()
{
    int sms = 0, clk = 0;
    CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    CHECK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0));
    printf("tmem_ld_rate sms %d max_clock_mhz %.0f\n", sms, clk / 1000.0);
    float* dout;
    CHECK(cudaMalloc(&dout, (size_t)sms * 16 * 32 * 4));
    if (run<4>(sms, clk / 1000.0, dout)) return 1;
    if (run<8>(sms, clk / 1000.0, dout)) return 1;
    if (run<16>(sms, clk / 1000.0, dout)) return 1;
    if (run_mma(sms, clk / 1000.0, 1, 1)) return 1;
    if (run_mma(sms, clk / 1000.0, 2, 1)) return 1;
    if (run_mma(sms, clk / 1000.0, 1, 2)) return 1;
    CHECK(cudaFree(dout));
    return 0;
}
