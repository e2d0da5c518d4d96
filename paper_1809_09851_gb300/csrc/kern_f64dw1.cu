// kern_f64dw1.cu -- the dim-1 building-block kernels for double storage computed
// in double-word (float-float) arithmetic, with native FP64 for out-of-range
// points.  One translation unit per dim keeps each compilation short.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_f64dw_d1(const LaunchReq& r, const KArgs& a) { return dispatch_dim<1, double, dw>(r, a); }
unsigned int wait_timeouts_f64dw_d1() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
