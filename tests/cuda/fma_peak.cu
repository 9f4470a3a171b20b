// fma_peak.cu -- measured FMA throughput of this GPU, the denominator of the
// FP32 screen's roofline next to the one derived from unit counts and clocks.
//
// Each thread runs kChains independent dependency chains of fused multiply-adds
// (scalar fma.rn.f32, packed fma.rn.f32x2 = two FP32 FMAs per instruction, and
// fma.rn.f64 for context) for kIters iterations; the grid is 8 CTAs of 256
// threads per SM.  Time with CUDA events around the timed launch (after one
// warm-up launch); flops = 2 per FMA lane.  The chains' final values are written
// out so that the loop cannot be removed.  Prints one line per kind:
//   fma_peak <kind> <TFLOP/s> <ms>
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kBlock = 256;

__global__ void fma_f32(float* out, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fma_f32x2(float* out, float a, float b)
{
    uint64_t x[kChains], av, bv;
    asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b), "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float lo = (float)(threadIdx.x + c), hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fma_f64(double* out, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < kIters / 8; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

#define CHECK(x)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) {                                                        \
            fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                    \
            return 1;                                                                   \
        }                                                                               \
    } while (0)

int main()
{
    int sms = 0, clk = 0;
    CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const int blocks = 8 * sms;
    const long long threads = (long long)blocks * kBlock;
    float* outf = nullptr;
    double* outd = nullptr;
    CHECK(cudaMalloc(&outf, sizeof(float) * threads));
    CHECK(cudaMalloc(&outd, sizeof(double) * threads));
    cudaEvent_t e0, e1;
    CHECK(cudaEventCreate(&e0));
    CHECK(cudaEventCreate(&e1));
    const float a = 0.999f, b = 0.001f;
    for (int kind = 0; kind < 3; ++kind) {
        for (int rep = 0; rep < 2; ++rep) {
            CHECK(cudaEventRecord(e0));
            if (kind == 0) fma_f32<<<blocks, kBlock>>>(outf, a, b);
            if (kind == 1) fma_f32x2<<<blocks, kBlock>>>(outf, a, b);
            if (kind == 2) fma_f64<<<blocks, kBlock>>>(outd, 0.999, 0.001);
            CHECK(cudaGetLastError());
            CHECK(cudaEventRecord(e1));
            CHECK(cudaEventSynchronize(e1));
            if (rep == 1) {
                float ms = 0.f;
                CHECK(cudaEventElapsedTime(&ms, e0, e1));
                const double lanes = kind == 1 ? 2.0 : 1.0;
                const double iters = kind == 2 ? kIters / 8 : kIters;
                const double flops = 2.0 * lanes * kChains * iters * (double)threads;
                const char* name = kind == 0 ? "f32" : (kind == 1 ? "f32x2" : "f64");
                printf("fma_peak %s %.3f %.4f\n", name, flops / (ms * 1e-3) / 1e12, ms);
            }
        }
    }
    CHECK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0));
    printf("fma_peak sms %d max_clock_mhz %.0f\n", sms, clk / 1000.0);
    cudaFree(outf);
    cudaFree(outd);
    return 0;
}
