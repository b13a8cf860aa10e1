// double instantiation of the per-sample 2D kernels (persample2d.cuh).
#include "persample2d.cuh"

namespace gs {
template gs_status launch_interp2d<double>(Plan*, PrecData<double>&, const double2*, double2*, const int32_t*, cudaStream_t,
                                           double*, const double2*, bool);
template gs_status launch_spread2d<double>(Plan*, PrecData<double>&, const double2*, const int32_t*, double2*, cudaStream_t);
}  // namespace gs
