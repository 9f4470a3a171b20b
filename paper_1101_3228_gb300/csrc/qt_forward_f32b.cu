// FP32-screen instantiations, dimension classes 6..16.
#include "qt_forward_launch.cuh"
namespace qt {
cudaError_t launch_f32_large(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                             cudaStream_t st)
{
#define QT_CASE(D, SS) \
    if (dm == D && S == SS) return launch_forward<D, SS, kF32Recheck, false>(p, block, dyn, num_sms, bps, st);
    QT_CASE(6, 1) QT_CASE(6, 2) QT_CASE(6, 4)
    QT_CASE(8, 1) QT_CASE(8, 2) QT_CASE(8, 4)
    QT_CASE(10, 1) QT_CASE(10, 2) QT_CASE(10, 4)
    QT_CASE(12, 1) QT_CASE(12, 2) QT_CASE(12, 4)
    QT_CASE(16, 1) QT_CASE(16, 2)
#undef QT_CASE
    return cudaErrorInvalidValue;
}
}  // namespace qt
