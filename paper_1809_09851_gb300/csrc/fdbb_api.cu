// fdbb_api.cu -- the C ABI declared in include/fdbb.h: argument checks,
// parameter-block assembly and dispatch to the per-storage-type kernels.
#include <atomic>
#include <cmath>
#include <cstdint>

#include "fdbb.h"
#include "fdbb_internal.h"

namespace fdbb {

int current_device_slot() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return dev >= 0 && dev < kMaxDevices ? dev : -1;
}

int device_sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const bool cached = dev >= 0 && dev < kMaxDevices;
  if (cached) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  if (cached) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

namespace {
thread_local fdbb_launch_info t_last_launch = {};
std::atomic<int> g_wait_limit{-1};
}  // namespace

void record_launch(int kernel, int grid, int block, int smem_bytes, int points_per_thread) {
  t_last_launch.kernel = kernel;
  t_last_launch.grid = grid;
  t_last_launch.block = block;
  t_last_launch.smem_bytes = smem_bytes;
  t_last_launch.points_per_thread = points_per_thread;
  t_last_launch.reserved = 0;
}

int wait_limit_setting() { return g_wait_limit.load(std::memory_order_relaxed); }

#ifdef FDBB_DEBUG
// Index-check counters of debug builds: violations, first bad index.
static __device__ unsigned long long g_debug_counters[2];

unsigned long long* debug_counters() {
  static std::atomic<unsigned long long*> cache[kMaxDevices];
  const int slot = current_device_slot();
  if (slot >= 0) {
    unsigned long long* p = cache[slot].load(std::memory_order_relaxed);
    if (p) return p;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_debug_counters) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (slot >= 0) cache[slot].store(static_cast<unsigned long long*>(p), std::memory_order_relaxed);
  return static_cast<unsigned long long*>(p);
}
#else
unsigned long long* debug_counters() { return nullptr; }
#endif

}  // namespace fdbb

namespace {

using fdbb::KArgs;
using fdbb::LaunchReq;
using fdbb::OpKind;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

fdbb_status check_dims(int dim, int64_t n) {
  if (dim < 1 || dim > 3 || n < 0) return FDBB_ERR_ARG;
  return FDBB_OK;
}

fdbb_status check_gamma(double gamma) {
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return FDBB_ERR_ARG;
  return FDBB_OK;
}

fdbb_status check_dtype(fdbb_dtype t) {
  return (t == FDBB_F64 || t == FDBB_F32 || t == FDBB_F16 || t == FDBB_BF16 || t == FDBB_F64_DW) ? FDBB_OK
                                                                                                  : FDBB_ERR_DTYPE;
}

// Required input planes: the array and every entry non-NULL and aligned.
fdbb_status take_in(KArgs& a, int base, const void* const* P, int k) {
  if (P == nullptr) return FDBB_ERR_NULLPTR;
  for (int i = 0; i < k; ++i) {
    if (P[i] == nullptr) return FDBB_ERR_NULLPTR;
    if (!aligned16(P[i])) return FDBB_ERR_ALIGN;
    a.in[base + i] = P[i];
  }
  return FDBB_OK;
}

// Optional output planes: a NULL array (when allowed) or NULL entries are
// skipped; non-NULL entries must be aligned.
fdbb_status take_out(KArgs& a, int base, void* const* P, int k, bool array_may_be_null) {
  if (P == nullptr) return array_may_be_null ? FDBB_OK : FDBB_ERR_NULLPTR;
  for (int i = 0; i < k; ++i) {
    if (P[i] != nullptr && !aligned16(P[i])) return FDBB_ERR_ALIGN;
    a.out[base + i] = P[i];
  }
  return FDBB_OK;
}

fdbb_status take_out1(KArgs& a, int slot, void* p) {
  if (p != nullptr && !aligned16(p)) return FDBB_ERR_ALIGN;
  a.out[slot] = p;
  return FDBB_OK;
}

// cv: specific heat at constant volume for the temperature (0: R = 1, i.e.
// c_v = 1/(gamma - 1)).
KArgs make_args(int64_t n, double gamma, double cv = 0.0) {
  KArgs a = {};
  a.n = n;
  const int polls = fdbb::wait_limit_setting();
  a.wait_override = polls < 0 ? 0 : polls + 1;
#ifdef FDBB_DEBUG
  a.dbg = fdbb::debug_counters();
#endif
  const double g = gamma, a1 = gamma - 1.0;
  const double tcv = cv > 0.0 ? 1.0 / (a1 * cv) : 1.0;
  const double kd[8] = {g, a1, 3.0 - g, 2.0 / a1, 1.0 / a1, -g, g / a1, tcv};
  for (int i = 0; i < 8; ++i) {
    a.kd[i] = kd[i];
    a.kf[i] = static_cast<float>(kd[i]);
    a.kl[i] = static_cast<float>(kd[i] - static_cast<double>(a.kf[i]));
  }
  return a;
}

// General EOS parameters into the kernel's EOS slots (double, and rounded
// once to float).  The model has been validated.
void set_eos_args(KArgs& a, const fdbb_eos_model& m) {
  const double a1 = m.gamma - 1.0;
  const double ke[8] = {a1, 1.0 / a1, m.b, 1.0 / m.cv, m.p_inf, m.q, m.gamma * m.p_inf, m.a};
  for (int i = 0; i < 8; ++i) {
    a.ke[i] = ke[i];
    a.kef[i] = static_cast<float>(ke[i]);
    a.kel[i] = static_cast<float>(ke[i] - static_cast<double>(a.kef[i]));
  }
}

// The double-word form needs every EOS parameter 0 or of magnitude in
// [2^-24, 2^24] (the range of its fast path); otherwise IEEE double is used.
bool eos_args_dw_range(const KArgs& a) {
  for (int i = 0; i < 8; ++i) {
    const double x = std::fabs(a.ke[i]);
    if (x != 0.0 && !(x >= 0x1p-24 && x <= 0x1p24)) return false;
  }
  return true;
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

fdbb_status check_eos(const fdbb_eos_model* m) {
  if (m == nullptr) return FDBB_ERR_ARG;
  if (m->kind != FDBB_EOS_IDEAL && m->kind != FDBB_EOS_NASG && m->kind != FDBB_EOS_VDW) return FDBB_ERR_ARG;
  if (m->reserved != 0) return FDBB_ERR_ARG;
  if (!(m->gamma > 1.0) || !std::isfinite(m->gamma)) return FDBB_ERR_ARG;
  if (!(m->cv > 0.0) || !std::isfinite(m->cv)) return FDBB_ERR_ARG;
  if (!finite_nonneg(m->b) || !std::isfinite(m->q)) return FDBB_ERR_ARG;
  if (m->kind == FDBB_EOS_NASG && !finite_nonneg(m->p_inf)) return FDBB_ERR_ARG;
  if (m->kind == FDBB_EOS_VDW && !finite_nonneg(m->a)) return FDBB_ERR_ARG;
  return FDBB_OK;
}

// Double-word general-EOS kernels, by model and dim.
cudaError_t dispatch_eos_f64dw(const LaunchReq& r, const KArgs& a) {
  using fdbb::EosKind;
  const bool nasg = r.eos == EosKind::Nasg;
  if (r.eos != EosKind::Nasg && r.eos != EosKind::Vdw) return cudaErrorInvalidValue;
  switch (r.dim) {
    case 1: return nasg ? fdbb::dispatch_eos_f64dw_nasg1(r, a) : fdbb::dispatch_eos_f64dw_vdw1(r, a);
    case 2: return nasg ? fdbb::dispatch_eos_f64dw_nasg2(r, a) : fdbb::dispatch_eos_f64dw_vdw2(r, a);
    case 3: return nasg ? fdbb::dispatch_eos_f64dw_nasg3(r, a) : fdbb::dispatch_eos_f64dw_vdw3(r, a);
    default: return cudaErrorInvalidValue;
  }
}

// Launch op for storage type t under the equation of state `eos`.
fdbb_status launch(fdbb_dtype t, OpKind op, int dim, int dir, KArgs& a, fdbb_stream_t stream,
                   fdbb::EosKind eos = fdbb::EosKind::Ideal) {
  if (a.n == 0) return FDBB_OK;
  a.nin = 0;
  while (a.nin < fdbb::kMaxIn && a.in[a.nin] != nullptr) ++a.nin;
  LaunchReq r{op, dim, dir, reinterpret_cast<cudaStream_t>(stream)};
  r.eos = eos;
  cudaError_t e = cudaErrorInvalidValue;
  if (eos != fdbb::EosKind::Ideal) {
    switch (t) {
      case FDBB_F64: e = fdbb::dispatch_eos_f64(r, a); break;
      case FDBB_F64_DW: e = eos_args_dw_range(a) ? dispatch_eos_f64dw(r, a) : fdbb::dispatch_eos_f64(r, a); break;
      case FDBB_F32: e = fdbb::dispatch_eos_f32(r, a); break;
      case FDBB_F16: e = fdbb::dispatch_eos_f16(r, a); break;
      case FDBB_BF16: e = fdbb::dispatch_eos_bf16(r, a); break;
      default: return FDBB_ERR_DTYPE;
    }
  } else {
    switch (t) {
      case FDBB_F64: e = fdbb::dispatch_f64(r, a); break;
      case FDBB_F32: e = fdbb::dispatch_f32(r, a); break;
      case FDBB_F16: e = fdbb::dispatch_f16(r, a); break;
      case FDBB_BF16: e = fdbb::dispatch_bf16(r, a); break;
      case FDBB_F64_DW:
        e = r.dim == 1 ? fdbb::dispatch_f64dw_d1(r, a)
            : r.dim == 2 ? fdbb::dispatch_f64dw_d2(r, a)
                         : fdbb::dispatch_f64dw_d3(r, a);
        break;
    }
  }
  return e == cudaSuccess ? FDBB_OK : FDBB_ERR_CUDA;
}


#define FDBB_TRY(expr)                   \
  do {                                   \
    const fdbb_status s_ = (expr);       \
    if (s_ != FDBB_OK) return s_;        \
  } while (0)

// Plane bookkeeping of each block, shared by the ideal-gas and general-EOS
// entry points: fills a.in / a.out from the caller's plane arrays.
fdbb_status fill_prim(KArgs& a, int dim, const void* const* U, void* const* V) {
  const int nv = dim + 2;
  FDBB_TRY(take_in(a, 0, U, nv));
  FDBB_TRY(take_out(a, 0, V, nv, false));
  if (a.out[0] == a.in[0]) a.out[0] = nullptr;  // rho onto itself: no copy
  return FDBB_OK;
}

fdbb_status fill_pc(KArgs& a, int dim, const void* const* U, void* p, void* c) {
  FDBB_TRY(take_in(a, 0, U, dim + 2));
  FDBB_TRY(take_out1(a, 0, p));
  return take_out1(a, 1, c);
}

fdbb_status fill_flux(KArgs& a, int dim, int dir, const void* const* U, void* const* F) {
  const int nv = dim + 2;
  FDBB_TRY(take_in(a, 0, U, nv));
  return take_out(a, 0, F, dir < 0 ? dim * nv : nv, false);
}

fdbb_status fill_jac(KArgs& a, int dim, const void* const* U, void* const* A) {
  const int nv = dim + 2;
  FDBB_TRY(take_in(a, 0, U, nv));
  return take_out(a, 0, A, nv * nv, false);
}

// Two nv-plane inputs (U and W, G or U_R), one nv-plane output.
fdbb_status fill_two(KArgs& a, int dim, const void* const* U, const void* const* W, void* const* Y) {
  const int nv = dim + 2;
  FDBB_TRY(take_in(a, 0, U, nv));
  FDBB_TRY(take_in(a, nv, W, nv));
  return take_out(a, 0, Y, nv, false);
}

fdbb_status fill_fused(KArgs& a, int dim, const void* const* U, const void* const* W, void* const* F,
                       void* const* A, void* const* Y) {
  const int nv = dim + 2;
  FDBB_TRY(take_in(a, 0, U, nv));
  FDBB_TRY(take_out(a, 0, F, dim * nv, true));
  FDBB_TRY(take_out(a, dim * nv, A, nv * nv, true));
  FDBB_TRY(take_out(a, dim * nv + nv * nv, Y, nv, true));
  bool want_y = false;
  for (int i = 0; i < nv; ++i) want_y = want_y || a.out[dim * nv + nv * nv + i] != nullptr;
  // W is read only when Y is wanted; otherwise in[nv] stays NULL.
  if (want_y) FDBB_TRY(take_in(a, nv, W, nv));
  return FDBB_OK;
}

fdbb_status fill_temp(KArgs& a, int dim, const void* const* U, void* T) {
  FDBB_TRY(take_in(a, 0, U, dim + 2));
  if (T == nullptr) return FDBB_ERR_NULLPTR;
  return take_out1(a, 0, T);
}

bool dir_ok(int dim, int dir, bool all_allowed) { return dir >= (all_allowed ? -1 : 0) && dir < dim; }

// Common checks and parameter block of a general-EOS entry point.  Sets
// `ideal` when the model is the ideal gas (the caller then forwards to the
// ideal-gas entry point, which checks the rest).
fdbb_status eos_prologue(const fdbb_eos_model* eos, int dim, int64_t n, fdbb_dtype t, KArgs& a, bool& ideal) {
  FDBB_TRY(check_dims(dim, n));
  FDBB_TRY(check_eos(eos));
  FDBB_TRY(check_dtype(t));
  ideal = eos->kind == FDBB_EOS_IDEAL;
  if (ideal) return FDBB_OK;
  a = make_args(n, eos->gamma, eos->cv);
  set_eos_args(a, *eos);
  return FDBB_OK;
}

fdbb::EosKind eos_kind(const fdbb_eos_model* eos) {
  return eos->kind == FDBB_EOS_NASG ? fdbb::EosKind::Nasg : fdbb::EosKind::Vdw;
}

}  // namespace

extern "C" {

const char* fdbb_status_string(fdbb_status s) {
  switch (s) {
    case FDBB_OK: return "ok";
    case FDBB_ERR_ARG: return "invalid argument (dim, dir, n, gamma or EOS model)";
    case FDBB_ERR_NULLPTR: return "required plane pointer is NULL";
    case FDBB_ERR_ALIGN: return "plane pointer is not 16-byte aligned";
    case FDBB_ERR_DTYPE: return "unknown storage type, or one the block does not support";
    case FDBB_ERR_CUDA: return "CUDA launch failed";
    case FDBB_ERR_TIMEOUT: return "timed out waiting for the device";
    case FDBB_ERR_NOMEM: return "buffer or memory budget too small";
  }
  return "unknown status";
}

int fdbb_version(void) { return 200; }

fdbb_ptr_kind fdbb_pointer_kind(const void* p) {
  if (p == nullptr) return FDBB_PTR_OTHER;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return FDBB_PTR_OTHER;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return FDBB_PTR_OTHER;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice: return at.device == cur ? FDBB_PTR_DEVICE : FDBB_PTR_OTHER;
    case cudaMemoryTypeManaged: return FDBB_PTR_MANAGED;
    case cudaMemoryTypeHost: return at.devicePointer == p ? FDBB_PTR_HOST : FDBB_PTR_OTHER;
    default: return FDBB_PTR_OTHER;
  }
}

fdbb_status fdbb_device_status(void) {
  const unsigned int n = fdbb::wait_timeouts_f64() + fdbb::wait_timeouts_f32() + fdbb::wait_timeouts_f16() +
                         fdbb::wait_timeouts_bf16() + fdbb::wait_timeouts_f64dw_d1() +
                         fdbb::wait_timeouts_f64dw_d2() + fdbb::wait_timeouts_f64dw_d3() +
                         fdbb::wait_timeouts_eos_f64() + fdbb::wait_timeouts_eos_f32() +
                         fdbb::wait_timeouts_eos_f16() + fdbb::wait_timeouts_eos_bf16() +
                         fdbb::wait_timeouts_eos_f64dw_nasg1() + fdbb::wait_timeouts_eos_f64dw_nasg2() +
                         fdbb::wait_timeouts_eos_f64dw_nasg3() + fdbb::wait_timeouts_eos_f64dw_vdw1() +
                         fdbb::wait_timeouts_eos_f64dw_vdw2() + fdbb::wait_timeouts_eos_f64dw_vdw3();
  return n ? FDBB_ERR_TIMEOUT : FDBB_OK;
}

int fdbb_set_wait_limit(int polls) {
  return fdbb::g_wait_limit.exchange(polls < 0 ? -1 : polls, std::memory_order_relaxed);
}

int64_t fdbb_debug_index_faults(int64_t* first_index) {
#ifdef FDBB_DEBUG
  unsigned long long* p = fdbb::debug_counters();
  if (p == nullptr) return -2;
  unsigned long long h[2] = {0, 0};
  if (cudaMemcpy(h, p, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  const unsigned long long zero[2] = {0, 0};
  if (h[0] != 0 && cudaMemcpy(p, zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess) cudaGetLastError();
  if (first_index) *first_index = h[0] ? static_cast<int64_t>(h[1]) : -1;
  return static_cast<int64_t>(h[0]);
#else
  if (first_index) *first_index = -1;
  return -1;
#endif
}

fdbb_status fdbb_last_launch(fdbb_launch_info* info) {
  if (info == nullptr) return FDBB_ERR_NULLPTR;
  *info = fdbb::t_last_launch;
  return FDBB_OK;
}

fdbb_status fdbb_v_mag2(int dim, int64_t n, fdbb_dtype t, const void* const* U, void* y, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, 1.4);
  FDBB_TRY(take_in(a, 0, U, dim + 1));
  if (y == nullptr) return FDBB_ERR_NULLPTR;
  FDBB_TRY(take_out1(a, 0, y));
  return launch(t, OpKind::VMag2, dim, 0, a, stream);
}

fdbb_status fdbb_prim_from_cons(int dim, double gamma, int64_t n, fdbb_dtype t, const void* const* U,
                                void* const* V, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_prim(a, dim, U, V));
  return launch(t, OpKind::Prim, dim, 0, a, stream);
}

fdbb_status fdbb_cons_from_prim(int dim, double gamma, int64_t n, fdbb_dtype t, const void* const* V,
                                void* const* U, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_prim(a, dim, V, U));
  return launch(t, OpKind::Cons, dim, 0, a, stream);
}

fdbb_status fdbb_eos(int dim, double gamma, int64_t n, fdbb_dtype t, const void* const* U, void* p, void* c,
                     fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_pc(a, dim, U, p, c));
  if (p == nullptr && c == nullptr) return FDBB_OK;
  return launch(t, OpKind::Eos, dim, 0, a, stream);
}

fdbb_status fdbb_riemann_inv(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, const void* const* U,
                             void* wm, void* wp, void* s, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(take_in(a, 0, U, dim + 2));
  FDBB_TRY(take_out1(a, 0, wm));
  FDBB_TRY(take_out1(a, 1, wp));
  FDBB_TRY(take_out1(a, 2, s));
  if (wm == nullptr && wp == nullptr && s == nullptr) return FDBB_OK;
  return launch(t, OpKind::Riemann, dim, dir, a, stream);
}

fdbb_status fdbb_flux(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, const void* const* U,
                      void* const* F, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, true)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_flux(a, dim, dir, U, F));
  return launch(t, dir < 0 ? OpKind::FluxAll : OpKind::Flux, dim, dir, a, stream);
}

fdbb_status fdbb_flux_jac(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, const void* const* U,
                          void* const* A, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_jac(a, dim, U, A));
  return launch(t, OpKind::Jac, dim, dir, a, stream);
}

fdbb_status fdbb_char_transform(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, int inverse,
                                const void* const* U, const void* const* W, void* const* Y,
                                fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_two(a, dim, U, W, Y));
  return launch(t, inverse ? OpKind::CharInv : OpKind::CharFwd, dim, dir, a, stream);
}

fdbb_status fdbb_euler_fused(int dim, int dir_jac, double gamma, int64_t n, fdbb_dtype t, const void* const* U,
                             const void* const* W, void* const* F, void* const* A, void* const* Y,
                             fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir_jac, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_fused(a, dim, U, W, F, A, Y));
  return launch(t, OpKind::Fused, dim, dir_jac, a, stream);
}

fdbb_status fdbb_euler_fused_host(int dim, int dir_jac, double gamma, int64_t n, fdbb_dtype t,
                                  const void* const* U, const void* const* W, void* const* F, void* const* A,
                                  void* const* Y, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir_jac, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_fused(a, dim, U, W, F, A, Y));
  if (n == 0) return FDBB_OK;
  for (int i = 0; i < fdbb::kMaxIn; ++i) {
    if (a.in[i] == nullptr) continue;
    const fdbb_ptr_kind k = fdbb_pointer_kind(a.in[i]);
    if (k == FDBB_PTR_OTHER) return FDBB_ERR_ARG;
    if (k != FDBB_PTR_DEVICE) a.flags |= fdbb::kDirectOnly;
  }
  for (int i = 0; i < fdbb::kMaxOut; ++i)
    if (a.out[i] != nullptr && fdbb_pointer_kind(a.out[i]) == FDBB_PTR_OTHER) return FDBB_ERR_ARG;
  return launch(t, OpKind::Fused, dim, dir_jac, a, stream);
}

fdbb_status fdbb_flux_prim(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, const void* const* V,
                           void* const* F, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, true)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_flux(a, dim, dir, V, F));
  return launch(t, dir < 0 ? OpKind::FluxPrimAll : OpKind::FluxPrim, dim, dir, a, stream);
}

fdbb_status fdbb_flux_jac_prim(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, const void* const* V,
                               void* const* B, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_jac(a, dim, V, B));
  return launch(t, OpKind::JacPrim, dim, dir, a, stream);
}

fdbb_status fdbb_temperature(int dim, double gamma, double cv, int64_t n, fdbb_dtype t, const void* const* U,
                             void* T, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  FDBB_TRY(check_gamma(gamma));
  if (!(cv > 0.0) || !std::isfinite(cv)) return FDBB_ERR_ARG;
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma, cv);
  FDBB_TRY(fill_temp(a, dim, U, T));
  return launch(t, OpKind::Temp, dim, 0, a, stream);
}

fdbb_status fdbb_roe_flux(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, const void* const* UL,
                          const void* const* UR, void* const* F, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_two(a, dim, UL, UR, F));
  return launch(t, OpKind::RoeFlux, dim, dir, a, stream);
}

fdbb_status fdbb_roe_char_transform(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, int inverse,
                                    const void* const* UL, const void* const* UR, const void* const* W,
                                    void* const* Y, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  const int nv = dim + 2;
  FDBB_TRY(take_in(a, 0, UL, nv));
  FDBB_TRY(take_in(a, nv, UR, nv));
  FDBB_TRY(take_in(a, 2 * nv, W, nv));
  FDBB_TRY(take_out(a, 0, Y, nv, false));
  return launch(t, inverse ? OpKind::RoeCharInv : OpKind::RoeCharFwd, dim, dir, a, stream);
}

fdbb_status fdbb_flux_vjp(int dim, int dir, double gamma, int64_t n, fdbb_dtype t, const void* const* U,
                          const void* const* G, void* const* gU, fdbb_stream_t stream) {
  FDBB_TRY(check_dims(dim, n));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  FDBB_TRY(check_gamma(gamma));
  FDBB_TRY(check_dtype(t));
  KArgs a = make_args(n, gamma);
  FDBB_TRY(fill_two(a, dim, U, G, gU));
  return launch(t, OpKind::Vjp, dim, dir, a, stream);
}

// ---------------------------------------------------------------------------
// General equations of state
// ---------------------------------------------------------------------------

fdbb_status fdbb_prim_from_cons_eos(const fdbb_eos_model* eos, int dim, int64_t n, fdbb_dtype t,
                                    const void* const* U, void* const* V, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (ideal) return fdbb_prim_from_cons(dim, eos->gamma, n, t, U, V, stream);
  FDBB_TRY(fill_prim(a, dim, U, V));
  return launch(t, OpKind::Prim, dim, 0, a, stream, eos_kind(eos));
}

fdbb_status fdbb_cons_from_prim_eos(const fdbb_eos_model* eos, int dim, int64_t n, fdbb_dtype t,
                                    const void* const* V, void* const* U, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (ideal) return fdbb_cons_from_prim(dim, eos->gamma, n, t, V, U, stream);
  FDBB_TRY(fill_prim(a, dim, V, U));
  return launch(t, OpKind::Cons, dim, 0, a, stream, eos_kind(eos));
}

fdbb_status fdbb_pressure_eos(const fdbb_eos_model* eos, int dim, int64_t n, fdbb_dtype t, const void* const* U,
                              void* p, void* c, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (ideal) return fdbb_eos(dim, eos->gamma, n, t, U, p, c, stream);
  FDBB_TRY(fill_pc(a, dim, U, p, c));
  if (p == nullptr && c == nullptr) return FDBB_OK;
  return launch(t, OpKind::Eos, dim, 0, a, stream, eos_kind(eos));
}

fdbb_status fdbb_temperature_eos(const fdbb_eos_model* eos, int dim, int64_t n, fdbb_dtype t,
                                 const void* const* U, void* T, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (ideal) return fdbb_temperature(dim, eos->gamma, eos->cv, n, t, U, T, stream);
  FDBB_TRY(fill_temp(a, dim, U, T));
  return launch(t, OpKind::Temp, dim, 0, a, stream, eos_kind(eos));
}

fdbb_status fdbb_flux_eos(const fdbb_eos_model* eos, int dim, int dir, int64_t n, fdbb_dtype t,
                          const void* const* U, void* const* F, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (!dir_ok(dim, dir, true)) return FDBB_ERR_ARG;
  if (ideal) return fdbb_flux(dim, dir, eos->gamma, n, t, U, F, stream);
  FDBB_TRY(fill_flux(a, dim, dir, U, F));
  return launch(t, dir < 0 ? OpKind::FluxAll : OpKind::Flux, dim, dir, a, stream, eos_kind(eos));
}

fdbb_status fdbb_flux_jac_eos(const fdbb_eos_model* eos, int dim, int dir, int64_t n, fdbb_dtype t,
                              const void* const* U, void* const* A, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  if (ideal) return fdbb_flux_jac(dim, dir, eos->gamma, n, t, U, A, stream);
  FDBB_TRY(fill_jac(a, dim, U, A));
  return launch(t, OpKind::Jac, dim, dir, a, stream, eos_kind(eos));
}

fdbb_status fdbb_char_transform_eos(const fdbb_eos_model* eos, int dim, int dir, int64_t n, fdbb_dtype t,
                                    int inverse, const void* const* U, const void* const* W, void* const* Y,
                                    fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  if (ideal) return fdbb_char_transform(dim, dir, eos->gamma, n, t, inverse, U, W, Y, stream);
  FDBB_TRY(fill_two(a, dim, U, W, Y));
  return launch(t, inverse ? OpKind::CharInv : OpKind::CharFwd, dim, dir, a, stream, eos_kind(eos));
}

fdbb_status fdbb_euler_fused_eos(const fdbb_eos_model* eos, int dim, int dir_jac, int64_t n, fdbb_dtype t,
                                 const void* const* U, const void* const* W, void* const* F, void* const* A,
                                 void* const* Y, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (!dir_ok(dim, dir_jac, false)) return FDBB_ERR_ARG;
  if (ideal) return fdbb_euler_fused(dim, dir_jac, eos->gamma, n, t, U, W, F, A, Y, stream);
  FDBB_TRY(fill_fused(a, dim, U, W, F, A, Y));
  return launch(t, OpKind::Fused, dim, dir_jac, a, stream, eos_kind(eos));
}

fdbb_status fdbb_flux_vjp_eos(const fdbb_eos_model* eos, int dim, int dir, int64_t n, fdbb_dtype t,
                              const void* const* U, const void* const* G, void* const* gU, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  if (ideal) return fdbb_flux_vjp(dim, dir, eos->gamma, n, t, U, G, gU, stream);
  FDBB_TRY(fill_two(a, dim, U, G, gU));
  return launch(t, OpKind::Vjp, dim, dir, a, stream, eos_kind(eos));
}

fdbb_status fdbb_flux_prim_eos(const fdbb_eos_model* eos, int dim, int dir, int64_t n, fdbb_dtype t,
                               const void* const* V, void* const* F, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (!dir_ok(dim, dir, true)) return FDBB_ERR_ARG;
  if (ideal) return fdbb_flux_prim(dim, dir, eos->gamma, n, t, V, F, stream);
  FDBB_TRY(fill_flux(a, dim, dir, V, F));
  return launch(t, dir < 0 ? OpKind::FluxPrimAll : OpKind::FluxPrim, dim, dir, a, stream, eos_kind(eos));
}

fdbb_status fdbb_flux_jac_prim_eos(const fdbb_eos_model* eos, int dim, int dir, int64_t n, fdbb_dtype t,
                                   const void* const* V, void* const* B, fdbb_stream_t stream) {
  KArgs a = {};
  bool ideal = false;
  FDBB_TRY(eos_prologue(eos, dim, n, t, a, ideal));
  if (!dir_ok(dim, dir, false)) return FDBB_ERR_ARG;
  if (ideal) return fdbb_flux_jac_prim(dim, dir, eos->gamma, n, t, V, B, stream);
  FDBB_TRY(fill_jac(a, dim, V, B));
  return launch(t, OpKind::JacPrim, dim, dir, a, stream, eos_kind(eos));
}

}  // extern "C"
