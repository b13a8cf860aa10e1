// float instantiation of the per-sample 2D kernels (persample2d.cuh).
#include "persample2d.cuh"

namespace gs {
template gs_status launch_interp2d<float>(Plan*, PrecData<float>&, const float2*, float2*, const int32_t*, cudaStream_t,
                                           double*, const float2*, bool);
template gs_status launch_spread2d<float>(Plan*, PrecData<float>&, const float2*, const int32_t*, float2*, cudaStream_t);
}  // namespace gs
