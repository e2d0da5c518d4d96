// kern_eos_f64.cu -- building-block kernels under the general EOS models, double storage.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_eos_f64(const LaunchReq& r, const KArgs& a) { return dispatch_eos<double, double>(r, a); }
unsigned int wait_timeouts_eos_f64() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
