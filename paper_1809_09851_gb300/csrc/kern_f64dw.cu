// kern_f64dw.cu -- all building-block kernels for double storage computed in
// double-word (float-float) arithmetic, with native FP64 for out-of-range points.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_f64dw(const LaunchReq& r, const KArgs& a) { return dispatch<double, dw>(r, a); }
unsigned int wait_timeouts_f64dw() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
