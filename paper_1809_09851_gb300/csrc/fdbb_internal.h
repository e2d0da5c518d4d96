// fdbb_internal.h -- types shared by the C-ABI layer and the kernel
// translation units (not part of the public interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdbb {

constexpr int kMaxIn = 15;   // U (nv) + W or G (nv); U_L, U_R, W (3 nv) for the Roe transform
constexpr int kMaxOut = 45;  // fused 3D: 15 flux + 25 Jacobian + 5 characteristic

enum class OpKind { VMag2, Prim, Cons, Eos, Riemann, Flux, FluxAll, Jac, CharFwd, CharInv, Fused, Vjp, RoeFlux,
                    RoeCharFwd, RoeCharInv, FluxPrim, FluxPrimAll, JacPrim, Temp };

// KArgs::flags: run the direct kernel (plain global loads) even where the
// staged one (bulk copies into shared memory) would be chosen -- for inputs in
// host memory, which the kernels read over the CPU-GPU link.
constexpr int kDirectOnly = 1;

// Kernel parameter block (passed by value as a __grid_constant__).
struct KArgs {
  const void* in[kMaxIn];
  void* out[kMaxOut];
  int64_t n;
  int nin;       // input planes in use (the leading non-NULL entries of in[])
  int flags;     // launch options (kDirectOnly); not read by the kernels
  int wait_override;  // staged kernels' polls per bounded wait: 0 = the default
                      // limit, k > 0 = k - 1 polls (fdbb_set_wait_limit)
  unsigned long long* dbg;  // debug builds: index-check counters (count, first bad index); else NULL
  double kd[8];  // gamma, gamma-1, 3-gamma, 2/(gamma-1), 1/(gamma-1), -gamma,
                 // gamma/(gamma-1), 1/((gamma-1) c_v)
  float kf[8];   // the same, rounded once to float
  float kl[8];   // kd - kf rounded to float: (kf, kl) is the double-word constant
  double ke[8];  // general EOS parameters (slots: gamma-1, 1/(gamma-1), b, 1/c_v,
                 // p_inf, q, gamma p_inf, a); unused by the ideal-gas kernels
  float kef[8];  // the same, rounded once to float
  float kel[8];  // ke - kef rounded to float: (kef, kel) is the double-word parameter
};

// Equation of state of a launch: the ideal gas (gamma in kd/kf/kl) or one of
// the general models (parameters in ke/kef).
enum class EosKind { Ideal = 0, Nasg = 1, Vdw = 2 };

struct LaunchReq {
  OpKind op;
  int dim;
  int dir;
  cudaStream_t stream;
  EosKind eos = EosKind::Ideal;
};

// Streaming multiprocessors of the current device (cached per device).
int device_sm_count();

// The current device, for per-device caches of kMaxDevices entries (-1 when
// it cannot be read or lies beyond the caches; callers then do not cache).
constexpr int kMaxDevices = 64;
int current_device_slot();

// Host-side record of the calling thread's last point-wise launch
// (fdbb_last_launch): kernel kind 1 = direct, 2 = staged.
void record_launch(int kernel, int grid, int block, int smem_bytes, int points_per_thread);

// Poll limit for the staged kernels' bounded waits (fdbb_set_wait_limit;
// < 0: the kernels' default).
int wait_limit_setting();

// Debug builds (FDBB_DEBUG): device address of the index-check counters on
// the current device (NULL if it cannot be looked up); release builds: NULL.
unsigned long long* debug_counters();

// Device-side index check of debug builds: true if `ok`; otherwise counts the
// violation in dbg[0], keeps the first bad index in dbg[1] and returns false,
// so that the caller skips the access.  Release builds compile it to true.
#ifdef FDBB_DEBUG
__device__ __forceinline__ bool dbg_check(unsigned long long* dbg, bool ok, int64_t index) {
  if (!ok && dbg != nullptr) {
    if (atomicAdd(&dbg[0], 1ull) == 0ull) dbg[1] = static_cast<unsigned long long>(index);
  }
  return ok;
}
#define FDBB_IDX_OK(dbg, cond, index) ::fdbb::dbg_check((dbg), (cond), (index))
#else
#define FDBB_IDX_OK(dbg, cond, index) true
#endif

// Defined once per storage type (one translation unit each).
cudaError_t dispatch_f64(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_f32(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_f16(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_bf16(const LaunchReq& r, const KArgs& a);
// (double-word: one translation unit per dim)
cudaError_t dispatch_f64dw_d1(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_f64dw_d2(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_f64dw_d3(const LaunchReq& r, const KArgs& a);
// General-EOS blocks (r.eos != Ideal): double storage in IEEE double and in
// double-word arithmetic, float / half / bfloat16 storage in float.
cudaError_t dispatch_eos_f64(const LaunchReq& r, const KArgs& a);
// (double-word: one translation unit per model and dim)
cudaError_t dispatch_eos_f64dw_nasg1(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_f64dw_nasg2(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_f64dw_nasg3(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_f64dw_vdw1(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_f64dw_vdw2(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_f64dw_vdw3(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_f32(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_f16(const LaunchReq& r, const KArgs& a);
cudaError_t dispatch_eos_bf16(const LaunchReq& r, const KArgs& a);

// Bounded device waits that ran out since the last call, per translation unit
// (read and cleared; synchronous).
unsigned int wait_timeouts_f64();
unsigned int wait_timeouts_f32();
unsigned int wait_timeouts_f16();
unsigned int wait_timeouts_bf16();
unsigned int wait_timeouts_f64dw_d1();
unsigned int wait_timeouts_f64dw_d2();
unsigned int wait_timeouts_f64dw_d3();
unsigned int wait_timeouts_eos_f64();
unsigned int wait_timeouts_eos_f64dw_nasg1();
unsigned int wait_timeouts_eos_f64dw_nasg2();
unsigned int wait_timeouts_eos_f64dw_nasg3();
unsigned int wait_timeouts_eos_f64dw_vdw1();
unsigned int wait_timeouts_eos_f64dw_vdw2();
unsigned int wait_timeouts_eos_f64dw_vdw3();
unsigned int wait_timeouts_eos_f32();
unsigned int wait_timeouts_eos_f16();
unsigned int wait_timeouts_eos_bf16();

}  // namespace fdbb
