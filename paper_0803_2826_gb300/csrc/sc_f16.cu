// Stream-collide instantiations for f16 population storage.
#include "stream_collide.cuh"

namespace lbi {
template cudaError_t launch_stream_collide_dt<1>(const lb_handle *, const void *, void *, const float *, float *);
template cudaError_t launch_patch_dt<1>(const lb_handle *, const void *, void *, float *, const int *, int,
                                         int, int, unsigned int *, unsigned int);
}  // namespace lbi
