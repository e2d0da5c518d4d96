// fdbb_device.cuh -- device-side building blocks: storage traits, vector
// streaming I/O, and the per-point Euler algebra.
//
// Each kernel thread owns VW consecutive points (one 128-bit word per plane for
// 2 x f64 or 4 x f32, one 64-bit word for 4 x f16/bf16), loads every input
// plane once, evaluates the
// requested expressions in registers and stores every output plane once.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdbb_dw.cuh"

namespace fdbb {

// ---------------------------------------------------------------------------
// Storage traits: register type L that a plane of storage type T is loaded
// into (double or float), and vector width VW (points per thread and plane).
// The compute type R is a separate kernel parameter: L itself, or the
// double-word type dw for double storage.
// ---------------------------------------------------------------------------
template <class T> struct Storage;
template <> struct Storage<double> { using L = double; static constexpr int VW = 2; };
template <> struct Storage<float> { using L = float; static constexpr int VW = 4; };
// 16-bit storage moves 64 bits (4 points) per plane and thread: 8 points of
// state would need ~150 registers and cap occupancy at one block per SM.
template <> struct Storage<__half> { using L = float; static constexpr int VW = 4; };
template <> struct Storage<__nv_bfloat16> { using L = float; static constexpr int VW = 4; };

// Points per thread and plane for storage T computed in R: the storage's
// vector width, except double-word, whose values take twice the registers of
// float and which therefore moves one double (64 bits) per plane and thread.
template <class T, class R> struct Width { static constexpr int VW = Storage<T>::VW; };
template <> struct Width<double, dw> { static constexpr int VW = 1; };

// Register type of one compute value's storage word: Storage<T>::L, except for
// packed double-word values (two points), whose storage word is a double pair.
struct fl2;  // two float points in one packed register pair (below)
template <class T, class R> struct LoadOf { using type = typename Storage<T>::L; };
template <> struct LoadOf<double, dw2> { using type = double2; };
template <class T> struct LoadOf<T, fl2> { using type = float2; };

// Double-word compute types, scalar or packed (they keep the loaded doubles of
// the outputs that are exact copies of inputs).
template <class R> struct IsDw { static constexpr bool value = false; };
template <> struct IsDw<dw> { static constexpr bool value = true; };
template <> struct IsDw<dw2> { static constexpr bool value = true; };

__device__ __forceinline__ double to_r(double x) { return x; }
__device__ __forceinline__ float to_r(float x) { return x; }
__device__ __forceinline__ float to_r(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_r(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class T> __device__ __forceinline__ T from_r(typename Storage<T>::L x);
template <> __device__ __forceinline__ double from_r<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_r<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_r<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_r<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}

// Vector streaming loads (evict-first: every input is touched once).
__device__ __forceinline__ void ld_vec(const double* p, double (&x)[1]) { x[0] = __ldcs(p); }
__device__ __forceinline__ void ld_vec(const double* p, double (&x)[2]) {
  double2 v = __ldcs(reinterpret_cast<const double2*>(p));
  x[0] = v.x;
  x[1] = v.y;
}
__device__ __forceinline__ void ld_vec(const float* p, float (&x)[4]) {
  float4 v = __ldcs(reinterpret_cast<const float4*>(p));
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
__device__ __forceinline__ void ld_vec(const __half* p, float (&x)[4]) {
  uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
  const uint32_t w[2] = {v.x, v.y};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    __half2 h = *reinterpret_cast<const __half2*>(&w[k]);
    float2 f = __half22float2(h);
    x[2 * k] = f.x;
    x[2 * k + 1] = f.y;
  }
}
__device__ __forceinline__ void ld_vec(const __nv_bfloat16* p, float (&x)[4]) {
  uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
  const uint32_t w[2] = {v.x, v.y};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[k]);
    float2 f = __bfloat1622float2(h);
    x[2 * k] = f.x;
    x[2 * k + 1] = f.y;
  }
}

// Vector streaming stores.
// (Evict-first: A/B on the double-word fused pass at 2^26, 13.60 Gpoints/s
// against 13.54 with write-back or L2-only stores.)
__device__ __forceinline__ void st_d2(double2* p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_vec(double* p, const double (&x)[1]) { __stcs(p, x[0]); }
__device__ __forceinline__ void st_vec(double* p, const double (&x)[2]) {
  st_d2(reinterpret_cast<double2*>(p), make_double2(x[0], x[1]));
}
__device__ __forceinline__ void st_vec(float* p, const float (&x)[4]) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
}
__device__ __forceinline__ void st_vec(__half* p, const float (&x)[4]) {
  uint32_t w[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    __half2 h = __floats2half2_rn(x[2 * k], x[2 * k + 1]);
    w[k] = *reinterpret_cast<uint32_t*>(&h);
  }
  __stcs(reinterpret_cast<uint2*>(p), make_uint2(w[0], w[1]));
}
__device__ __forceinline__ void st_vec(__nv_bfloat16* p, const float (&x)[4]) {
  uint32_t w[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * k], x[2 * k + 1]);
    w[k] = *reinterpret_cast<uint32_t*>(&h);
  }
  __stcs(reinterpret_cast<uint2*>(p), make_uint2(w[0], w[1]));
}

// Vector reads of a tile staged in shared memory (plain loads; the data was
// written there by the tensor-memory-access engine).
__device__ __forceinline__ void ld_sh(const double* p, double (&x)[1]) { x[0] = p[0]; }
__device__ __forceinline__ void ld_sh(const double* p, double (&x)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  x[0] = v.x;
  x[1] = v.y;
}
__device__ __forceinline__ void ld_sh(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
__device__ __forceinline__ void ld_sh(const __half* p, float (&x)[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  x[0] = a.x;
  x[1] = a.y;
  x[2] = b.x;
  x[3] = b.y;
}
__device__ __forceinline__ void ld_sh(const __nv_bfloat16* p, float (&x)[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
  x[0] = a.x;
  x[1] = a.y;
  x[2] = b.x;
  x[3] = b.y;
}

// Range guard of a compute type: a no-op for IEEE types; for dw it records
// whether every checked value lies in the double-word fast-path range.
struct NoGuard {
  static constexpr bool ok = true;
  template <class X> __device__ __forceinline__ void check(const X&) {}
};
template <class R> struct GuardOf { using type = NoGuard; };
template <> struct GuardOf<dw> { using type = DwGuard; };
template <> struct GuardOf<dw2> { using type = DwGuard2; };

// Register value (double or float) -> compute type.
template <class R, class G> __device__ __forceinline__ R to_compute(double x, G&) { return x; }
template <class R, class G> __device__ __forceinline__ R to_compute(float x, G&) { return x; }
template <> __device__ __forceinline__ dw to_compute<dw, DwGuard>(double x, DwGuard& g) {
  return dw_from_double(x, g);
}
template <class R, class G> __device__ __forceinline__ R to_compute(double2 x, G& g) { return dw2_from_double2(x, g); }
template <class R, class G> __device__ __forceinline__ R to_compute(float2 x, G&) { return R(x); }
// Compute type -> register value of the storage's load type.
__device__ __forceinline__ double to_load(double x) { return x; }
__device__ __forceinline__ float to_load(float x) { return x; }
__device__ __forceinline__ double to_load(dw x) { return dw_to_double(x); }
__device__ __forceinline__ double2 to_load(dw2 x) { return dw2_to_double2(x); }
__device__ __forceinline__ float2 to_load(const fl2& x);

// The same in conversion form C of the double-word types (fdbb_dw.cuh; the
// default form is the one of to_compute and to_load).
template <class R, DwConv C, class G, class L> __device__ __forceinline__ R to_compute_c(L x, G& g) {
  if constexpr (C != DwConv::kClamp && std::is_same<R, dw2>::value)
    return dw2_from_double2<C>(x, g);
  else if constexpr (C != DwConv::kClamp && std::is_same<R, dw>::value)
    return dw_from_double<C>(x, g);
  else
    return to_compute<R, G>(x, g);
}
template <DwConv C, class R> __device__ __forceinline__ auto to_load_c(const R& x) {
  if constexpr (C != DwConv::kClamp && std::is_same<R, dw2>::value)
    return dw2_to_double2<C>(x);
  else if constexpr (C != DwConv::kClamp && std::is_same<R, dw>::value)
    return dw_to_double<C>(x);
  else
    return to_load(x);
}

// Load VW points starting at i0 in the storage's load type; cnt < VW only in
// the ragged last chunk, where the missing lanes get `fill` (a harmless
// in-range value that is never stored).
template <class T, int VW>
__device__ __forceinline__ void load_raw(const T* p, int64_t i0, int cnt, typename Storage<T>::L (&raw)[VW],
                                         float fill) {
  using L = typename Storage<T>::L;
  if (cnt == VW) {
    ld_vec(p + i0, raw);
  } else {
#pragma unroll
    for (int j = 0; j < VW; ++j) raw[j] = (j < cnt) ? to_r(p[i0 + j]) : static_cast<L>(fill);
  }
}

// Load VW points and convert them to the compute type R.
template <class T, int VW, class R, class G>
__device__ __forceinline__ void load(const T* p, int64_t i0, int cnt, R (&x)[VW], float fill, G& g) {
  typename Storage<T>::L raw[VW];
  load_raw<T, VW>(p, i0, cnt, raw, fill);
#pragma unroll
  for (int j = 0; j < VW; ++j) x[j] = to_compute<R, G>(raw[j], g);
}

// Store VW values of the storage's load type; a NULL plane is skipped.
template <class T, int VW>
__device__ __forceinline__ void store_raw(T* p, int64_t i0, int cnt, const typename Storage<T>::L (&raw)[VW]) {
  if (p == nullptr) return;
  if (cnt == VW) {
    st_vec(p + i0, raw);
  } else {
#pragma unroll
    for (int j = 0; j < VW; ++j)
      if (j < cnt) p[i0 + j] = from_r<T>(raw[j]);
  }
}

// Store a pair of doubles (the two points of a packed value): cnt of them.
template <class T, int VW>
__device__ __forceinline__ void store_raw(T* p, int64_t i0, int cnt, const double2 (&raw)[VW]) {
  static_assert(VW == 1, "one pair per call");
  if (p == nullptr) return;
  if (cnt == 2) {
    st_d2(reinterpret_cast<double2*>(p + i0), raw[0]);
  } else if (cnt == 1) {
    p[i0] = raw[0].x;
  }
}

// Store pairs of float values (the points of packed float pairs): cnt points
// (all 2 VW of them, or the first cnt of a ragged last chunk).
template <class T, int VW>
__device__ __forceinline__ void store_raw(T* p, int64_t i0, int cnt, const float2 (&raw)[VW]) {
  if (p == nullptr) return;
  float x[2 * VW];
#pragma unroll
  for (int j = 0; j < VW; ++j) {
    x[2 * j] = raw[j].x;
    x[2 * j + 1] = raw[j].y;
  }
  if (cnt == 2 * VW) {
    st_vec(p + i0, x);
  } else {
#pragma unroll
    for (int j = 0; j < 2 * VW; ++j)
      if (j < cnt) p[i0 + j] = from_r<T>(x[j]);
  }
}

// Store VW points of the compute type; a NULL plane is skipped.
template <class T, int VW, class R>
__device__ __forceinline__ void store(T* p, int64_t i0, int cnt, const R (&x)[VW]) {
  if (p == nullptr) return;
  typename LoadOf<T, R>::type raw[VW];
#pragma unroll
  for (int j = 0; j < VW; ++j) raw[j] = to_load(x[j]);
  store_raw<T, VW>(p, i0, cnt, raw);
}

// store in conversion form C
template <class T, int VW, class R, DwConv C>
__device__ __forceinline__ void store_c(T* p, int64_t i0, int cnt, const R (&x)[VW]) {
  if (p == nullptr) return;
  typename LoadOf<T, R>::type raw[VW];
#pragma unroll
  for (int j = 0; j < VW; ++j) raw[j] = to_load_c<C>(x[j]);
  store_raw<T, VW>(p, i0, cnt, raw);
}

// ---------------------------------------------------------------------------
// Arithmetic helpers, overloaded on the compute type.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_(float x) { return 1.0f / x; }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double abs_(double x) { return fabs(x); }
__device__ __forceinline__ float abs_(float x) { return fabsf(x); }
__device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
// x/2 and 2x (exact scalings; double-word scales both words).
__device__ __forceinline__ double half_(double x) { return 0.5 * x; }
__device__ __forceinline__ float half_(float x) { return 0.5f * x; }
__device__ __forceinline__ dw half_(dw x) { return dw(__fmul_rn(0.5f, x.hi), __fmul_rn(0.5f, x.lo)); }
__device__ __forceinline__ double twice_(double x) { return x + x; }
__device__ __forceinline__ float twice_(float x) { return x + x; }
__device__ __forceinline__ dw twice_(dw x) { return dw(__fadd_rn(x.hi, x.hi), __fadd_rn(x.lo, x.lo)); }
__device__ __forceinline__ dw2 half_(dw2 x) { return dw2(p_mul(make_float2(0.5f, 0.5f), x.hi), p_mul(make_float2(0.5f, 0.5f), x.lo)); }
__device__ __forceinline__ dw2 twice_(dw2 x) { return dw2(p_add(x.hi, x.hi), p_add(x.lo, x.lo)); }

// ---------------------------------------------------------------------------
// Two float points in one packed FP32x2 register pair (sm_100 and later).  The
// float-arithmetic blocks (FP32, FP16 and BF16 storage) evaluate the four
// points of a thread as two such pairs: each addition, multiplication and
// FMA is one FADD2 / FMUL2 / FFMA2 for both points, rounded to nearest per
// lane; divisions, square roots, absolute values and powers run per lane.
// ---------------------------------------------------------------------------
struct fl2 {
  float2 v;
  fl2() = default;
  __device__ __forceinline__ constexpr fl2(float2 x) : v(x) {}
  __device__ __forceinline__ fl2(float x) : v(make_float2(x, x)) {}
  __device__ __forceinline__ fl2(int x) : v(make_float2(static_cast<float>(x), static_cast<float>(x))) {}
  fl2(double) = delete;
};
__device__ __forceinline__ fl2 operator+(fl2 a, fl2 b) { return fl2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ fl2 operator*(fl2 a, fl2 b) { return fl2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ fl2 operator-(fl2 a) { return fl2(make_float2(-a.v.x, -a.v.y)); }
// a - b as (-1) b + a: the product is exact, so one rounding as in a subtraction
__device__ __forceinline__ fl2 operator-(fl2 a, fl2 b) {
  return fl2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ fl2 fma_(fl2 a, fl2 b, fl2 c) { return fl2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ fl2 half_(fl2 x) { return fl2(__fmul2_rn(make_float2(0.5f, 0.5f), x.v)); }
__device__ __forceinline__ fl2 twice_(fl2 x) { return fl2(__fadd2_rn(x.v, x.v)); }
__device__ __forceinline__ fl2 rcp_(fl2 x) { return fl2(make_float2(1.0f / x.v.x, 1.0f / x.v.y)); }
__device__ __forceinline__ fl2 operator/(fl2 a, fl2 b) { return fl2(make_float2(a.v.x / b.v.x, a.v.y / b.v.y)); }
__device__ __forceinline__ fl2 rsqrt_(fl2 x) { return fl2(make_float2(rsqrtf(x.v.x), rsqrtf(x.v.y))); }
__device__ __forceinline__ fl2 sqrt_(fl2 x) { return fl2(make_float2(sqrtf(x.v.x), sqrtf(x.v.y))); }
__device__ __forceinline__ fl2 abs_(fl2 x) { return fl2(make_float2(fabsf(x.v.x), fabsf(x.v.y))); }
__device__ __forceinline__ fl2 pow_(fl2 x, fl2 y) { return fl2(make_float2(powf(x.v.x, y.v.x), powf(x.v.y, y.v.y))); }
__device__ __forceinline__ float2 to_load(const fl2& x) { return x.v; }

}  // namespace fdbb

// General EOS models and dual numbers (they use the arithmetic helpers above).
#include "fdbb_eos.cuh"

namespace fdbb {

// Constants derived from gamma on the host in double, rounded once to R: the
// ideal-gas model of the per-point formulas (general EOS models, whose
// kIdeal is false, live in fdbb_eos.cuh).
template <class R> struct Consts {
  static constexpr bool kIdeal = true;
  R g;      // gamma
  R a1;     // gamma - 1
  R g3;     // 3 - gamma
  R ta1;    // 2 / (gamma - 1)
  R ia1;    // 1 / (gamma - 1)
  R mg;     // -gamma
  R gia1;   // gamma / (gamma - 1)
  R tcv;    // 1 / ((gamma - 1) c_v): T = p / rho * tcv
};

// ---------------------------------------------------------------------------
// Per-point state
// ---------------------------------------------------------------------------
// The loaded doubles of rho and m, kept for the outputs that are exact copies
// of an input (F_d[0] = m_d, rho in cons <-> prim) when the compute type is
// double-word (whose split of a double keeps 47 of its 53 bits).
template <class R, int D> struct RawState {};
template <int D> struct RawState<dw, D> {
  double rho, m[D];
};
template <int D> struct RawState<dw2, D> {
  double2 rho, m[D];
};

template <class R, int D> struct Pt {
  RawState<R, D> raw;
  R rho, m[D], rE;  // conservative state
  R r;              // 1 / rho
  R v[D];           // velocity
  R rq;             // kinetic energy density rho |v|^2 / 2
  R q;              // |v|^2 / 2
  R p;              // pressure
  R H;              // total specific enthalpy (rhoE + p) / rho
  R c2;             // squared speed of sound gamma p / rho
  // General EOS only (the ideal-gas formulas use constants instead):
  R G;              // Grueneisen coefficient (1/rho) dp/de|_rho   (ideal: gamma - 1)
  R ph;             // dp/drho at constant m, rhoE                  (ideal: (gamma - 1) q)
  R ie;             // specific internal energy e
  R zr, zp;         // d(rho e)/drho|_p and d(rho e)/dp|_rho of the inverse rho e(rho, p)
};

// EOS-dependent coefficients of the Euler algebra: constants of the ideal
// gas, per-point values of a general EOS.
//   Gamma = (1/rho) dp/de, phi = dp/drho|_(m, rhoE) = dp/drho|_e + Gamma (q - e)
template <class R, int D, class K> __device__ __forceinline__ R eos_G(const Pt<R, D>& s, const K& k) {
  if constexpr (K::kIdeal) return k.a1; else return s.G;
}
template <class R, int D, class K> __device__ __forceinline__ R eos_phi(const Pt<R, D>& s, const K& k) {
  if constexpr (K::kIdeal) return k.a1 * s.q; else return s.ph;
}
template <class R, int D, class K> __device__ __forceinline__ R eos_1pG(const Pt<R, D>& s, const K& k) {
  if constexpr (K::kIdeal) return k.g; else return R(1) + s.G;  // 1 + Gamma
}
template <class R, int D, class K> __device__ __forceinline__ R eos_2mG(const Pt<R, D>& s, const K& k) {
  if constexpr (K::kIdeal) return k.g3; else return R(2) - s.G;  // 2 - Gamma
}

// Error-free transforms (Knuth TwoSum, FMA-based TwoProduct), written with
// round-to-nearest intrinsics so that no contraction or reassociation applies.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Internal-energy density rho e = rhoE - |m|^2 / (2 rho).
//  double, dw: plain evaluation (error ~ u * (rhoE + rho q)).
//  float : compensated evaluation; |m|^2 is summed exactly as a float pair
//          (TwoProduct + TwoSum, Ogita-Rump-Oishi), divided by 2 rho with a
//          remainder correction, and subtracted from rhoE with TwoSum, so the
//          result is accurate to a few ulp of rho e itself even when
//          rho q / rho e ~ 1e3 (Mach 50) or rho ~ 1e-4 (near vacuum).
template <class R, int D>
__device__ __forceinline__ void internal_energy(Pt<R, D>& s, R& rhoe) {
  R mv = s.m[0] * s.v[0];
#pragma unroll
  for (int i = 1; i < D; ++i) mv = fma_(s.m[i], s.v[i], mv);
  s.rq = half_(mv);
  rhoe = s.rE - s.rq;
}
template <int D>
__device__ __forceinline__ void internal_energy(Pt<float, D>& s, float& rhoe) {
  float hi, lo;
  two_prod(s.m[0], s.m[0], hi, lo);
#pragma unroll
  for (int i = 1; i < D; ++i) {
    float ph, pl, t;
    two_prod(s.m[i], s.m[i], ph, pl);
    two_sum(hi, ph, hi, t);
    lo = __fadd_rn(lo, __fadd_rn(t, pl));
  }
  hi = __fmul_rn(0.5f, hi);  // exact scaling by 1/2
  lo = __fmul_rn(0.5f, lo);
  const float qh = __fmul_rn(hi, s.r);           // rho q, leading part
  const float rem = __fmaf_rn(-qh, s.rho, hi);   // hi - qh rho (exact or nearly)
  const float ql = __fmul_rn(__fadd_rn(rem, lo), s.r);
  float d, t;
  two_sum(s.rE, -qh, d, t);
  rhoe = __fadd_rn(d, __fsub_rn(t, ql));
  s.rq = qh;
}
// The same compensated evaluation on packed pairs, each lane step for step
// the float one above.
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 bb = pk_sub(s, a);
  e = __fadd2_rn(pk_sub(a, pk_sub(s, bb)), pk_sub(b, bb));
}
__device__ __forceinline__ void two_prod2(float2 a, float2 b, float2& p, float2& e) {
  p = __fmul2_rn(a, b);
  e = __ffma2_rn(a, b, make_float2(-p.x, -p.y));
}
template <int D>
__device__ __forceinline__ void internal_energy(Pt<fl2, D>& s, fl2& rhoe) {
  float2 hi, lo;
  two_prod2(s.m[0].v, s.m[0].v, hi, lo);
#pragma unroll
  for (int i = 1; i < D; ++i) {
    float2 ph, pl, t;
    two_prod2(s.m[i].v, s.m[i].v, ph, pl);
    two_sum2(hi, ph, hi, t);
    lo = __fadd2_rn(lo, __fadd2_rn(t, pl));
  }
  const float2 h = make_float2(0.5f, 0.5f);
  hi = __fmul2_rn(h, hi);  // exact scaling by 1/2
  lo = __fmul2_rn(h, lo);
  const float2 qh = __fmul2_rn(hi, s.r.v);
  const float2 rem = __ffma2_rn(make_float2(-qh.x, -qh.y), s.rho.v, hi);
  const float2 ql = __fmul2_rn(__fadd2_rn(rem, lo), s.r.v);
  float2 d, t;
  two_sum2(s.rE.v, make_float2(-qh.x, -qh.y), d, t);
  rhoe = fl2(__fadd2_rn(d, pk_sub(t, ql)));
  s.rq = fl2(qh);
}

// Conservative -> derived state.  One reciprocal per point.  The guard sees
// every derived quantity that later enters a product (1/rho is covered by
// rho, 1/c and (gamma-1)/c^2 by c^2).
//
// A general EOS evaluates p(rho, e) once on dual numbers, which also gives
// dp/drho|_e and dp/de|_rho; then Gamma = (1/rho) dp/de,
// c^2 = dp/drho|_e + Gamma p / rho (the isentropic derivative, de = p/rho^2 drho)
// and phi = dp/drho|_e + Gamma (q - e).
// C2 = false skips c^2 (and its range check) for blocks that never read it:
// fluxes, Jacobians, the flux VJP, the Roe forms (which average their own).
// WH = false skips H and WQ = false skips q (each with its check) for blocks
// that do not read them: neither for EOS, Riemann invariants, the flux
// columns and the temperature; H for the forward characteristic transform;
// q for the two states of the Roe forms (a general EOS still forms q, for
// phi).  In double-word arithmetic at N = 2^26 on one GB300 (fraction of the
// measured HBM bandwidth, with / without the skips): EOS 0.91 / 0.82,
// Riemann invariants 0.82 / 0.75, temperature 0.93 / 0.83, one flux column
// 0.94 / 0.91, forward characteristic transform 0.88 / 0.84, Roe flux
// 0.32 / 0.32; cons -> prim 0.90 / 0.91 keeps them.
template <bool C2 = true, bool WH = true, bool WQ = WH, class R, int D, class K, class G>
__device__ __forceinline__ void derive(Pt<R, D>& s, const K& k, G& g) {
  constexpr bool kQ = WQ || !K::kIdeal;
  s.r = rcp_(s.rho);
#pragma unroll
  for (int i = 0; i < D; ++i) s.v[i] = s.m[i] * s.r;
  R rhoe;
  internal_energy(s, rhoe);
  if constexpr (kQ) s.q = s.rq * s.r;
  if constexpr (K::kIdeal) {
    s.p = k.a1 * rhoe;
    if constexpr (WH) s.H = (s.rE + s.p) * s.r;
    if constexpr (C2) s.c2 = k.g * s.p * s.r;
  } else {
    s.ie = rhoe * s.r;
    const D2<R> P = tangents(k.p_rhoe(arg1(s.rho), arg2(s.ie)));
    s.p = P.v;
    s.G = P.de * s.r;
    if constexpr (WH) s.H = (s.rE + s.p) * s.r;
    if constexpr (C2) s.c2 = fma_(s.G * s.p, s.r, P.dr);
    s.ph = fma_(s.G, s.q - s.ie, P.dr);
    g.check(s.ie);
    g.check(s.G);
    g.check(s.ph);
  }
#pragma unroll
  for (int i = 0; i < D; ++i) g.check(s.v[i]);
  if constexpr (kQ) g.check(s.q);
  g.check(s.p);
  if constexpr (WH) g.check(s.H);
  if constexpr (C2) g.check(s.c2);
}

// ---------------------------------------------------------------------------
// Per-point formulas.  `d` is a compile-time direction.
// ---------------------------------------------------------------------------

// Flux column d: F[0] = m_d, F[1+i] = m_d v_i + delta_id p, F[nv-1] = v_d (rhoE + p).
// For i != d, F_d[1+i] = F_i[1+d] = m_i m_d / rho; both are formed as
// m_min(i,d) v_max(i,d), so a pass over several directions computes (and
// converts) each such product once.
template <int D, int d, class R>
__device__ __forceinline__ R flux_comp(const Pt<R, D>& s, int k) {
  if (k == 0) return s.m[d];
  if (k == D + 1) return s.v[d] * (s.rE + s.p);
  const int i = k - 1;
  if (i == d) return fma_(s.m[d], s.v[d], s.p);
  return i < d ? s.m[i] * s.v[d] : s.m[d] * s.v[i];
}

// Jacobian entry A_d[row][col] (row-major), u = v_d, with dp/dU =
// (phi, -Gamma v, Gamma) (ideal gas: phi = (gamma-1) q, Gamma = gamma - 1).
template <int D, int d, class R, class K>
__device__ __forceinline__ R jac_entry(const Pt<R, D>& s, const K& k, int row, int col) {
  constexpr int nv = D + 2;
  const R u = s.v[d];
  if (row == 0) return (col == 1 + d) ? R(1) : R(0);
  if (row == nv - 1) {
    if (col == 0) return u * (eos_phi(s, k) - s.H);
    if (col == nv - 1) return eos_1pG(s, k) * u;
    if (col == 1 + d) return fma_(-(eos_G(s, k) * u), u, s.H);
    return -(eos_G(s, k) * u) * s.v[col - 1];
  }
  const int i = row - 1;
  if (i != d) {
    if (col == 0) return -(u * s.v[i]);
    if (col == 1 + d) return s.v[i];
    if (col == 1 + i) return u;
    return R(0);
  }
  // row 1 + d
  if (col == 0) return fma_(-u, u, eos_phi(s, k));
  if (col == nv - 1) return eos_G(s, k);
  if (col == 1 + d) return eos_2mG(s, k) * u;
  return -(eos_G(s, k) * s.v[col - 1]);
}

// Tangential direction t_k of d (ascending), compile-time.
template <int D, int d> __device__ __forceinline__ constexpr int tang(int k) {
  return (k < d) ? k : k + 1;
}

// Forward characteristic transform Y = L_d W at one point (see fdbb.h):
//   t = b1 (q w0 - v.w + w_e), a = (u w0 - w_d) / c, b1 = (gamma-1)/c^2
//   Y0 = (t + a)/2, Y1 = w0 - t, Y_{1+k} = w_{t_k} - v_{t_k} w0, Y_{nv-1} = (t - a)/2
// For a general EOS t = (dp/dU . w) / c^2 = (phi w0 + Gamma (w_e - v.w)) / c^2.
template <int D, int d, class R, class K>
__device__ __forceinline__ void char_fwd(const Pt<R, D>& s, const K& k, const R* w, R* y) {
  constexpr int nv = D + 2;
  const R ic = rsqrt_(s.c2);
  R dot = s.v[0] * w[1];
#pragma unroll
  for (int i = 1; i < D; ++i) dot = fma_(s.v[i], w[1 + i], dot);
  R t;
  if constexpr (K::kIdeal) {
    const R b1 = k.a1 * ic * ic;
    t = b1 * (fma_(s.q, w[0], w[nv - 1]) - dot);
  } else {
    t = fma_(s.ph, w[0], s.G * (w[nv - 1] - dot)) * (ic * ic);
  }
  const R a = fma_(s.v[d], w[0], -w[1 + d]) * ic;
  y[0] = half_(t + a);
  y[1] = w[0] - t;
#pragma unroll
  for (int kk = 0; kk < D - 1; ++kk) {
    const int tk = tang<D, d>(kk);
    y[2 + kk] = fma_(-s.v[tk], w[0], w[1 + tk]);
  }
  y[nv - 1] = half_(t - a);
}

// Inverse characteristic transform Y = R_d W at one point.  The entropy wave's
// energy component is q for the ideal gas and 2q - phi/Gamma for a general EOS
// (the value that leaves the pressure unchanged across the wave).
template <int D, int d, class R, class K>
__device__ __forceinline__ void char_inv_sums(const Pt<R, D>& s, const K& k, const R* w, R sum, R anm1, R a1pn,
                                              R* y) {
  constexpr int nv = D + 2;
  const R c = sqrt_(s.c2);
  const R a2 = w[1];
  const R dif = c * anm1;
  y[0] = sum;
#pragma unroll
  for (int i = 0; i < D; ++i) y[1 + i] = s.v[i] * sum;
  y[1 + d] = y[1 + d] + dif;
  R e = fma_(s.H, a1pn, s.v[d] * dif);
  if constexpr (K::kIdeal)
    e = fma_(s.q, a2, e);
  else
    e = fma_(twice_(s.q) - s.ph / s.G, a2, e);
#pragma unroll
  for (int kk = 0; kk < D - 1; ++kk) {
    const int tk = tang<D, d>(kk);
    y[1 + tk] = y[1 + tk] + w[2 + kk];
    e = fma_(s.v[tk], w[2 + kk], e);
  }
  y[nv - 1] = e;
}

// The same with the weight sums formed here, in R: for weights that are
// themselves computed (the Roe flux's wave strengths).
template <int D, int d, class R, class K>
__device__ __forceinline__ void char_inv(const Pt<R, D>& s, const K& k, const R* w, R* y) {
  constexpr int nv = D + 2;
  char_inv_sums<D, d>(s, k, w, w[0] + w[1] + w[nv - 1], w[nv - 1] - w[0], w[0] + w[nv - 1], y);
}

// gU = A_d^T G at one point, with z = g_d + u g_e and sigma = sum_{i != d} v_i g_i:
//   gU[0]     = phi z - u sigma - u (u g_d + H g_e)
//   gU[1+j]   = u g_j - (gamma-1) v_j z             (j != d)
//   gU[1+d]   = g_0 + sigma + 2 u g_d + H g_e - (gamma-1) u z
//   gU[nv-1]  = (gamma-1) g_d + gamma u g_e
// (general EOS: gamma - 1 -> Gamma, gamma -> 1 + Gamma, phi per point).
template <int D, int d, class R, class K>
__device__ __forceinline__ void flux_vjp_pt(const Pt<R, D>& s, const K& k, const R* g, R* y) {
  constexpr int nv = D + 2;
  const R u = s.v[d];
  const R gd = g[1 + d], ge = g[nv - 1];
  const R z = fma_(u, ge, gd);
  constexpr int t0 = d == 0 ? 1 : 0;  // first tangential direction
  R sigma = R(0);
#pragma unroll
  for (int i = 0; i < D; ++i)
    if (i != d) sigma = i == t0 ? s.v[i] * g[1 + i] : fma_(s.v[i], g[1 + i], sigma);
  const R phi = eos_phi(s, k), a1 = eos_G(s, k);
  y[0] = fma_(phi, z, -fma_(u, sigma, u * fma_(u, gd, s.H * ge)));
#pragma unroll
  for (int j = 0; j < D; ++j)
    if (j != d) y[1 + j] = fma_(u, g[1 + j], -(a1 * s.v[j] * z));
  y[1 + d] = g[0] + sigma + fma_(twice_(u), gd, fma_(s.H, ge, -(a1 * u * z)));
  y[nv - 1] = fma_(a1, gd, eos_1pG(s, k) * u * ge);
}

// State from primitive variables (rho, v, p set): m = rho v, q = |v|^2/2,
// rhoE = p/(gamma-1) + rho q (paper section 2.2, Fig. 9, the primitive form);
// for a general EOS rhoE = rho e(rho, p) + rho q, with the partial derivatives
// of rho e(rho, p) from one dual-number evaluation.
template <class R, int D, class K, class G>
__device__ __forceinline__ void derive_prim(Pt<R, D>& s, const K& k, G& g) {
  R v2 = s.v[0] * s.v[0];
#pragma unroll
  for (int i = 1; i < D; ++i) v2 = fma_(s.v[i], s.v[i], v2);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    s.m[i] = s.rho * s.v[i];
    g.check(s.m[i]);
  }
  s.q = half_(v2);
  s.rq = s.rho * s.q;
  if constexpr (K::kIdeal) {
    s.rE = fma_(s.p, k.ia1, s.rq);
  } else {
    const D2<R> Z = tangents(k.rhoe_rhop(arg1(s.rho), arg2(s.p)));
    s.rE = Z.v + s.rq;
    s.zr = Z.dr;
    s.zp = Z.de;
    g.check(s.zr);
    g.check(s.zp);
  }
  g.check(s.q);
  g.check(s.rE);
}

// Entry of B_d = dF_d/dV (rows in U order, columns in V order), u = v_d:
//   row 0: (u, rho at col 1+d, 0); row 1+i: (u v_i, rho (delta_jd v_i +
//   delta_ij u), delta_id); row nv-1: (u q, delta_jd (gamma/(gamma-1) p +
//   rho q) + rho u v_j, gamma/(gamma-1) u).  General EOS, with z = rho e(rho, p):
//   row nv-1: (u (q + dz/drho), delta_jd (rhoE + p) + rho u v_j, u (dz/dp + 1)).
template <int D, int d, class R, class K>
__device__ __forceinline__ R jacp_entry(const Pt<R, D>& s, const K& k, int row, int col) {
  constexpr int nv = D + 2;
  const R u = s.v[d];
  if (row == 0) return col == 0 ? u : (col == 1 + d ? s.rho : R(0));
  if (row == nv - 1) {
    if constexpr (K::kIdeal) {
      if (col == 0) return u * s.q;
      if (col == nv - 1) return k.gia1 * u;
      const R e = s.m[col - 1] * u;  // rho v_j u
      return col == 1 + d ? e + fma_(k.gia1, s.p, s.rq) : e;
    } else {
      if (col == 0) return u * (s.q + s.zr);
      if (col == nv - 1) return fma_(u, s.zp, u);
      const R e = s.m[col - 1] * u;
      return col == 1 + d ? e + (s.rE + s.p) : e;
    }
  }
  const int i = row - 1;
  if (col == 0) return u * s.v[i];
  if (col == nv - 1) return i == d ? R(1) : R(0);
  const int j = col - 1;
  if (j == d && j == i) return s.m[i] + s.rho * u;  // rho v_i + rho u
  if (j == d) return s.m[i];
  if (j == i) return s.rho * u;
  return R(0);
}

// Roe-averaged state of (L, R) (P. L. Roe, J. Comput. Phys. 43, 1981): with
// w = sqrt(rho), v^ = (w_L v_L + w_R v_R)/(w_L + w_R), H^ likewise,
// q^ = |v^|^2/2, c^2 = (gamma-1)(H^ - q^).  Sets the fields the
// characteristic formulas read (v, q, H, c2).
template <class R, int D, class G>
__device__ __forceinline__ void roe_state(const Pt<R, D>& L, const Pt<R, D>& Rt, const Consts<R>& k, Pt<R, D>& s,
                                          G& g) {
  const R wL = sqrt_(L.rho), wR = sqrt_(Rt.rho);
  const R iw = rcp_(wL + wR);
  R v2 = R(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    s.v[i] = fma_(wL, L.v[i], wR * Rt.v[i]) * iw;
    v2 = (i == 0) ? s.v[i] * s.v[i] : fma_(s.v[i], s.v[i], v2);
    g.check(s.v[i]);
  }
  s.H = fma_(wL, L.H, wR * Rt.H) * iw;
  s.q = half_(v2);
  s.c2 = k.a1 * (s.H - s.q);
  g.check(s.H);
  g.check(s.q);
  g.check(s.c2);
}

// Roe flux in direction d: (F_d(L) + F_d(R))/2 - 1/2 R^ (|lambda^| * (L^ (U_R - U_L))).
template <int D, int d, class R>
__device__ __forceinline__ void roe_flux_pt(const Pt<R, D>& L, const Pt<R, D>& Rt, const Pt<R, D>& s,
                                            const Consts<R>& k, R* Fh) {
  constexpr int nv = D + 2;
  R dU[nv], alpha[nv], beta[nv], diss[nv];
  dU[0] = Rt.rho - L.rho;
#pragma unroll
  for (int i = 0; i < D; ++i) dU[1 + i] = Rt.m[i] - L.m[i];
  dU[nv - 1] = Rt.rE - L.rE;
  char_fwd<D, d>(s, k, dU, alpha);
  const R u = s.v[d], c = sqrt_(s.c2);
  beta[0] = abs_(u - c) * alpha[0];
#pragma unroll
  for (int q = 1; q < nv - 1; ++q) beta[q] = abs_(u) * alpha[q];
  beta[nv - 1] = abs_(u + c) * alpha[nv - 1];
  char_inv<D, d>(s, k, beta, diss);
#pragma unroll
  for (int q = 0; q < nv; ++q)
    Fh[q] = half_(flux_comp<D, d>(L, q) + flux_comp<D, d>(Rt, q) - diss[q]);
}

}  // namespace fdbb
