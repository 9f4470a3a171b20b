// qt_forward_tc_in.cu -- instantiations of the tensor-core screen whose
// certifier warps draw the samples themselves (one launch per step; a unit of
// its own so that both layouts compile in parallel).
#include "qt_forward_tc.cuh"

namespace qt {

cudaError_t launch_tc_forward_drawin(int dm, const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st)
{
    if (dm == 2) return launch_tc<2, 1, true>(p, dyn, num_sms, bps, st);
    if (dm == 4) return launch_tc<4, 1, true>(p, dyn, num_sms, bps, st);
    if (dm == 6) return launch_tc<6, 2, true>(p, dyn, num_sms, bps, st);
    if (dm == 8) return launch_tc<8, 2, true>(p, dyn, num_sms, bps, st);
    if (dm == 10) return launch_tc<10, 2, true>(p, dyn, num_sms, bps, st);
    return cudaErrorInvalidValue;
}

}  // namespace qt
