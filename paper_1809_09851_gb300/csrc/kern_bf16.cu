// kern_bf16.cu -- all building-block kernels for __nv_bfloat16 storage.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_bf16(const LaunchReq& r, const KArgs& a) { return dispatch<__nv_bfloat16, float>(r, a); }
unsigned int wait_timeouts_bf16() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
