// kern_eos_f64dw_vdw1.cu -- the VDW model's building-block kernels for dim 1,
// double storage computed in double-word arithmetic (IEEE double for chunks
// outside its range).  One translation unit per (model, dim) keeps each
// compilation short.
#include "fdbb_kernels.cuh"

namespace fdbb {
cudaError_t dispatch_eos_f64dw_vdw1(const LaunchReq& r, const KArgs& a) {
  return dispatch_eos_dim<1, double, dw, VdwModel>(r, a);
}
unsigned int wait_timeouts_eos_f64dw_vdw1() { return take_wait_timeouts_tu(); }
}  // namespace fdbb
