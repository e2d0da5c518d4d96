// kern_eos_f32.cu -- building-block kernels under the general EOS models, float storage.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_eos_f32(const LaunchReq& r, const KArgs& a) { return dispatch_eos<float, float>(r, a); }
unsigned int wait_timeouts_eos_f32() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
