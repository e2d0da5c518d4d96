// kern_f32.cu -- all building-block kernels for float storage.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_f32(const LaunchReq& r, const KArgs& a) { return dispatch<float, float>(r, a); }
unsigned int wait_timeouts_f32() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
