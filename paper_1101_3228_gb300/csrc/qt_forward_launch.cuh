// qt_forward_launch.cuh -- launch helper shared by the instantiation units.
#pragma once
#include "qt_forward.cuh"

namespace qt {

template <int DM, int S, int FORM, bool STREAMED>
cudaError_t launch_forward(const ForwardParams& p, int block, int dyn, int num_sms, int* bps, cudaStream_t st)
{
    auto kern = forward_kernel<DM, S, FORM, STREAMED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, block, dyn);
    if (e != cudaSuccess) return e;
    if (b < 1) return cudaErrorInvalidConfiguration;
    *bps = b;
    long long grid = (long long)num_sms * b;
    if (grid > p.total_items) grid = p.total_items;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, dyn, st>>>(p);
    return cudaGetLastError();
}

}  // namespace qt
