// kern_f16.cu -- all building-block kernels for __half storage.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_f16(const LaunchReq& r, const KArgs& a) { return dispatch<__half, float>(r, a); }
unsigned int wait_timeouts_f16() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
