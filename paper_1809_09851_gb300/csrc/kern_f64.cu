// kern_f64.cu -- all building-block kernels for double storage.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_f64(const LaunchReq& r, const KArgs& a) { return dispatch<double, double>(r, a); }
unsigned int wait_timeouts_f64() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
