// kern_f32.cu -- all building-block kernels for float storage.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_f32(const LaunchReq& r, const KArgs& a) { return dispatch<float, float>(r, a); }
}  // namespace fdbb
