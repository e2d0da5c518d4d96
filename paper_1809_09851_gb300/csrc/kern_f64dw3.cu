// kern_f64dw3.cu -- the dim-3 building-block kernels for double storage computed
// in double-word (float-float) arithmetic, with native FP64 for out-of-range
// points.  One translation unit per dim keeps each compilation short.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_f64dw_d3(const LaunchReq& r, const KArgs& a) { return dispatch_dim<3, double, dw>(r, a); }
unsigned int wait_timeouts_f64dw_d3() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
