// tmem_ld_red.cu -- test program: the reduction form of the tensor-memory load
// (tcgen05.ld.red.32x32b.xN.{min,max}.f32) returns, per thread, the minimum
// (maximum) of the N columns it loads, and the loaded columns themselves.  The
// tensor-core screen takes its 16-column chunk minima from this instruction,
// so its certificate relies on that minimum being exact.
//
// One CTA of 128 threads allocates 32 TMEM columns, stores known values with
// tcgen05.st, reads them back with tcgen05.ld.red and frees the columns; the
// host compares against minima computed on the CPU.  Prints one summary line.
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <cuda_runtime.h>

__device__ __forceinline__ float val(int t, int c) { return (float)(((t * 37 + c * 101) % 257) - 128) + 0.03125f * (float)c; }

__global__ void probe(float* out)   // out: [128][4 + 32]
{
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(32u) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = s_tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t w[32];
    for (int c = 0; c < 32; ++c) w[c] = __float_as_uint(val(t, c));
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                 :: "r"(tm), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15]),
                    "r"(w[16]), "r"(w[17]), "r"(w[18]), "r"(w[19]), "r"(w[20]), "r"(w[21]), "r"(w[22]), "r"(w[23]), "r"(w[24]), "r"(w[25]), "r"(w[26]), "r"(w[27]), "r"(w[28]), "r"(w[29]), "r"(w[30]), "r"(w[31]) : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    float a[16], b[16], r0, r1, r2;
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, %16, [%17];"
                 : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7]), "=f"(a[8]), "=f"(a[9]), "=f"(a[10]), "=f"(a[11]), "=f"(a[12]), "=f"(a[13]), "=f"(a[14]), "=f"(a[15]), "=f"(r0)
                 : "r"(tm) : "memory");
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x16.min.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, %16, [%17];"
                 : "=f"(b[0]), "=f"(b[1]), "=f"(b[2]), "=f"(b[3]), "=f"(b[4]), "=f"(b[5]), "=f"(b[6]), "=f"(b[7]), "=f"(b[8]), "=f"(b[9]), "=f"(b[10]), "=f"(b[11]), "=f"(b[12]), "=f"(b[13]), "=f"(b[14]), "=f"(b[15]), "=f"(r1)
                 : "r"(tm + 16u) : "memory");
    float c32[32];
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"
                 : "=f"(c32[0]), "=f"(c32[1]), "=f"(c32[2]), "=f"(c32[3]), "=f"(c32[4]), "=f"(c32[5]), "=f"(c32[6]), "=f"(c32[7]), "=f"(c32[8]), "=f"(c32[9]), "=f"(c32[10]), "=f"(c32[11]), "=f"(c32[12]), "=f"(c32[13]), "=f"(c32[14]), "=f"(c32[15]),
                   "=f"(c32[16]), "=f"(c32[17]), "=f"(c32[18]), "=f"(c32[19]), "=f"(c32[20]), "=f"(c32[21]), "=f"(c32[22]), "=f"(c32[23]), "=f"(c32[24]), "=f"(c32[25]), "=f"(c32[26]), "=f"(c32[27]), "=f"(c32[28]), "=f"(c32[29]), "=f"(c32[30]), "=f"(c32[31]), "=f"(r2)
                 : "r"(tm) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    float* o = out + t * 36;
    o[0] = r0; o[1] = r1; o[2] = r2; o[3] = 0.f;
    for (int c = 0; c < 16; ++c) { o[4 + c] = a[c]; o[20 + c] = b[c]; }
    float diff = 0.f;
    for (int c = 0; c < 32; ++c) diff += fabsf(c32[c] - val(t, c));
    o[3] = diff;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(32u) : "memory");
}

static float hval(int t, int c) { return (float)(((t * 37 + c * 101) % 257) - 128) + 0.03125f * (float)c; }

int main()
{
    float* d;
    cudaMalloc(&d, 128 * 36 * 4);
    cudaMemset(d, 0, 128 * 36 * 4);
    probe<<<1, 128>>>(d);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("cuda error %s\n", cudaGetErrorString(e)); return 1; }
    float h[128 * 36];
    cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    int bad_min16a = 0, bad_min16b = 0, bad_max32 = 0, bad_vals = 0;
    for (int t = 0; t < 128; ++t) {
        float m0 = 1e30f, m1 = 1e30f, M = -1e30f;
        for (int c = 0; c < 16; ++c) m0 = fminf(m0, hval(t, c));
        for (int c = 16; c < 32; ++c) m1 = fminf(m1, hval(t, c));
        for (int c = 0; c < 32; ++c) M = fmaxf(M, hval(t, c));
        const float* o = h + t * 36;
        if (o[0] != m0) { if (bad_min16a < 4) printf("t=%d red16@0 %g expect %g\n", t, o[0], m0); ++bad_min16a; }
        if (o[1] != m1) { if (bad_min16b < 4) printf("t=%d red16@16 %g expect %g\n", t, o[1], m1); ++bad_min16b; }
        if (o[2] != M) { if (bad_max32 < 4) printf("t=%d red32max %g expect %g\n", t, o[2], M); ++bad_max32; }
        for (int c = 0; c < 16; ++c) if (o[4 + c] != hval(t, c) || o[20 + c] != hval(t, 16 + c)) ++bad_vals;
        if (o[3] != 0.f) ++bad_vals;
    }
    printf("ld.red probe: min16@0 bad %d, min16@16 bad %d, max32 bad %d, loaded values bad %d (of 128 rows)\n", bad_min16a, bad_min16b, bad_max32, bad_vals);
    printf("row0: red %g %g %g\n", h[0], h[1], h[2]);
    return 0;
}
