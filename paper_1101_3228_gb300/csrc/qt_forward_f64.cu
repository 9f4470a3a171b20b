// Plain FP64 instantiations (exact distances, every dimension class).
#include "qt_forward_launch.cuh"
#include "qt_launch.h"
namespace qt {
cudaError_t launch_f64(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                       cudaStream_t st)
{
#define QT_CASE(D, SS) \
    if (dm == D && S == SS) return launch_forward<D, SS, kPlainF64, false>(p, block, dyn, num_sms, bps, st);
    QT_CASE(1, 1) QT_CASE(1, 2) QT_CASE(1, 4)
    QT_CASE(2, 1) QT_CASE(2, 2) QT_CASE(2, 4)
    QT_CASE(3, 1) QT_CASE(3, 2)
    QT_CASE(4, 1) QT_CASE(4, 2)
    QT_CASE(6, 1) QT_CASE(8, 1) QT_CASE(10, 1) QT_CASE(12, 1) QT_CASE(16, 1)
#undef QT_CASE
    return cudaErrorInvalidValue;
}

static bool in_list(int dm, int S, const int (*tab)[2], int n)
{
    for (int i = 0; i < n; ++i)
        if (tab[i][0] == dm && tab[i][1] == S) return true;
    return false;
}

bool forward_variant_exists(int form, int dm, int S, bool streamed)
{
    static const int f32s[][2] = {{4, 1}, {4, 2}, {4, 4}, {6, 1}, {6, 2}, {6, 4}, {8, 1}, {8, 2}, {8, 4},
                                  {10, 1}, {10, 2}, {10, 4}, {12, 1}, {12, 2}, {16, 1}, {16, 2}};
    if (form == kTcRecheck) return S == 1 && (dm == 2 || dm == 4 || dm == 6 || dm == 8 || dm == 10);
    if (form == kRouterCert) return S == 1;
    if (streamed) return form == kF32Recheck && in_list(dm, S, f32s, (int)(sizeof f32s / sizeof f32s[0]));
    static const int f32[][2] = {{1, 2}, {1, 4}, {1, 8}, {2, 2}, {2, 4}, {2, 8}, {3, 2}, {3, 4}, {3, 8},
                                 {4, 2}, {4, 4}, {4, 8}, {6, 1}, {6, 2}, {6, 4}, {8, 1}, {8, 2}, {8, 4},
                                 {10, 1}, {10, 2}, {10, 4}, {12, 1}, {12, 2}, {12, 4}, {16, 1}, {16, 2}};
    static const int f64[][2] = {{1, 1}, {1, 2}, {1, 4}, {2, 1}, {2, 2}, {2, 4}, {3, 1}, {3, 2},
                                 {4, 1}, {4, 2}, {6, 1}, {8, 1}, {10, 1}, {12, 1}, {16, 1}};
    if (form == kF32Recheck) return in_list(dm, S, f32, (int)(sizeof f32 / sizeof f32[0]));
    if (form == kPlainF64) return in_list(dm, S, f64, (int)(sizeof f64 / sizeof f64[0]));
    return false;
}

cudaError_t forward_launch(int form, int dm, int S, bool streamed, const ForwardParams& p, int block, int dyn_smem,
                           int num_sms, int* blocks_per_sm, cudaStream_t st)
{
    if (form == kTcRecheck) return launch_tc_forward(dm, p, dyn_smem, num_sms, blocks_per_sm, st);
    if (form == kRouterCert) return launch_router_forward(dm, p, num_sms, blocks_per_sm, st);
    if (form == kPathwise)
        return launch_pathwise(dm, S, p.prec == 1, streamed, p, dyn_smem, num_sms, blocks_per_sm, st);
    if (streamed) {
        if (form != kF32Recheck) return cudaErrorInvalidValue;
        return launch_f32_streamed(dm, S, p, block, dyn_smem, num_sms, blocks_per_sm, st);
    }
    if (form == kPlainF64) return launch_f64(dm, S, p, block, dyn_smem, num_sms, blocks_per_sm, st);
    if (form == kF32Recheck) {
        if (dm <= 4) return launch_f32_small(dm, S, p, block, dyn_smem, num_sms, blocks_per_sm, st);
        return launch_f32_large(dm, S, p, block, dyn_smem, num_sms, blocks_per_sm, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace qt
