// kern_eos_f16.cu -- building-block kernels under the general EOS models,
// __half storage computed in float (compensated internal energy).
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_eos_f16(const LaunchReq& r, const KArgs& a) { return dispatch_eos<__half, float>(r, a); }
unsigned int wait_timeouts_eos_f16() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
