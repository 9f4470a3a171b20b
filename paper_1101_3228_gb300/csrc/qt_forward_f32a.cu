// FP32-screen instantiations, dimension classes 1..4.
#include "qt_forward_launch.cuh"
namespace qt {
cudaError_t launch_f32_small(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                             cudaStream_t st)
{
#define QT_CASE(D, SS) \
    if (dm == D && S == SS) return launch_forward<D, SS, kF32Recheck, false>(p, block, dyn, num_sms, bps, st);
    QT_CASE(1, 2) QT_CASE(1, 4) QT_CASE(1, 8)
    QT_CASE(2, 2) QT_CASE(2, 4) QT_CASE(2, 8)
    QT_CASE(3, 2) QT_CASE(3, 4) QT_CASE(3, 8)
    QT_CASE(4, 2) QT_CASE(4, 4) QT_CASE(4, 8)
#undef QT_CASE
    return cudaErrorInvalidValue;
}
}  // namespace qt
