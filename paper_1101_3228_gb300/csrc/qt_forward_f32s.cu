// FP32-screen instantiations of the streamed-grid mode (grids larger than
// one CTA's shared memory pass through a two-slot ring of bulk copies).
#include "qt_forward_launch.cuh"
#include "qt_launch.h"
namespace qt {
cudaError_t launch_f32_streamed(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                                cudaStream_t st)
{
#define QT_CASE(D, SS) \
    if (dm == D && S == SS) return launch_forward<D, SS, kF32Recheck, true>(p, block, dyn, num_sms, bps, st);
    QT_CASE(4, 1) QT_CASE(4, 2) QT_CASE(4, 4)
    QT_CASE(6, 1) QT_CASE(6, 2) QT_CASE(6, 4)
    QT_CASE(8, 1) QT_CASE(8, 2) QT_CASE(8, 4)
    QT_CASE(10, 1) QT_CASE(10, 2) QT_CASE(10, 4)
    QT_CASE(12, 1) QT_CASE(12, 2)
    QT_CASE(16, 1) QT_CASE(16, 2)
#undef QT_CASE
    return cudaErrorInvalidValue;
}
}  // namespace qt
