// kern_eos_bf16.cu -- building-block kernels under the general EOS models,
// __nv_bfloat16 storage computed in float (compensated internal energy).
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_eos_bf16(const LaunchReq& r, const KArgs& a) { return dispatch_eos<__nv_bfloat16, float>(r, a); }
unsigned int wait_timeouts_eos_bf16() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
