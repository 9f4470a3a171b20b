// qt_launch.h -- dispatch from run-time (form, dimension class, samples per
// thread) to the compiled instantiations of the forward kernel.
#pragma once
#include <cuda_runtime.h>

#include "qt_internal.h"

namespace qt {

bool forward_variant_exists(int form, int dm, int S, bool streamed);

// Launches one persistent grid (SM count x resident CTAs per SM).
cudaError_t forward_launch(int form, int dm, int S, bool streamed, const ForwardParams& p, int block, int dyn_smem,
                           int num_sms, int* blocks_per_sm, cudaStream_t st);

// per-file dispatchers (qt_forward_*.cu)
cudaError_t launch_f32_small(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                             cudaStream_t st);
cudaError_t launch_f32_large(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                             cudaStream_t st);
cudaError_t launch_f64(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                       cudaStream_t st);
cudaError_t launch_router_forward(int dm, const ForwardParams& p, int num_sms, int* bps, cudaStream_t st);
cudaError_t launch_tc_forward(int dm, const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st);
cudaError_t launch_tc_forward_drawin(int dm, const ForwardParams& p, int dyn, int num_sms, int* bps, cudaStream_t st);
// draw pass of the tensor-core form over the items [p.item_lo, p.item_hi)
cudaError_t launch_tc_draw(int dm, const ForwardParams& p, cudaStream_t st);
// Algorithm II (path-wise): compiled variants, default paths per thread, launch
bool pathwise_variant_exists(int dm, int S, bool f32, bool streamed);
int pathwise_default_spt(int dm, bool f32, bool streamed, long long M, long long ctas);
cudaError_t launch_pathwise(int dm, int S, bool f32, bool streamed, const ForwardParams& p, int dyn, int num_sms,
                            int* bps, cudaStream_t st);
cudaError_t launch_f32_streamed(int dm, int S, const ForwardParams& p, int block, int dyn, int num_sms, int* bps,
                                cudaStream_t st);

}  // namespace qt
