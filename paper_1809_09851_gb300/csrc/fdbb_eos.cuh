// fdbb_eos.cuh -- general equations of state for the building-block kernels.
//
// The paper lets a user plug in an equation of state of the form f(p, V, T) = 0
// by writing a type with static members p_rhoe(rho, e) and T_rhoe(rho, e)
// (section 2.2, "Equations of state", Fig. 10).  Here an EOS model is a small
// device struct with the same members plus the inverse rhoe_rhop(rho, p):
//
//   template <class X, class Y> auto p_rhoe(const X& rho, const Y& e) const;   // pressure
//   R T_rhoe(R rho, R e) const;                                                 // temperature
//   template <class X, class Y> auto rhoe_rhop(const X& rho, const Y& p) const; // rho e
//
// p_rhoe and rhoe_rhop are templates over the number types so that the
// kernels can evaluate them on forward-mode dual numbers (D2 below) and get the
// partial derivatives the flux Jacobians and eigenvectors need -- dp/drho at
// constant e, dp/de at constant rho, and those of rho e(rho, p) -- exactly, from
// the one formula the model writes.  `kIdeal = false` routes the per-point
// formulas (fdbb_device.cuh) to their general-EOS forms.
//
// This header is included by fdbb_device.cuh after the arithmetic helpers
// (rcp_, fma_, ...) that the dual numbers use.
//
// Adding an EOS: write such a struct (parameters are the members, filled from
// the eight slots of the kernel's EOS parameter block), give it a model tag
// with `make`, and list it in the EOS dispatcher (kern_eos_*.cu).
#pragma once

#include "fdbb_dw.cuh"
#include "fdbb_internal.h"

namespace fdbb {

// Forward-mode dual number with two tangents: value v and the derivatives with
// respect to the first (dr) and second (de) argument of the evaluated function.
// Each tangent also has a kind known at compile time -- exactly zero, exactly
// one, or a run-time value -- and only kVal tangents are stored.  The seeds of
// the two arguments are (1, 0) and (0, 1); propagating the kinds drops every
// product with an exact zero or one from the derivative formulas (under IEEE
// rules the compiler may not fold x * 0, and x * 1 still costs a double-word
// product), so a model's derivatives cost only their nonzero terms.
enum TangentKind : int { kZero = 0, kOne = 1, kVal = 2 };

template <class R, int KR = kVal, int KE = kVal> struct D2 {
  R v, dr, de;  // dr (de) holds a value only when KR (KE) is kVal
};

namespace dual {
// Tangent x of kind K as a number.
template <int K, class R> __device__ __forceinline__ R val(const R& x) {
  if constexpr (K == kZero) return R(0);
  else if constexpr (K == kOne) return R(1);
  else return x;
}
__host__ __device__ constexpr int add_kind(int a, int b) { return a == kZero ? b : (b == kZero ? a : kVal); }
__host__ __device__ constexpr int neg_kind(int a) { return a == kZero ? kZero : kVal; }
__host__ __device__ constexpr int sub_kind(int a, int b) { return b == kZero ? a : (a == kZero ? neg_kind(b) : kVal); }
__host__ __device__ constexpr int scale_kind(int a) { return a == kZero ? kZero : kVal; }

// a + b, a - b and -a for tangents of kinds A and B (results of kinds
// add_kind, sub_kind and neg_kind).
template <int A, int B, class R> __device__ __forceinline__ R add(const R& a, const R& b) {
  if constexpr (A == kZero) return b;
  else if constexpr (B == kZero) return a;
  else return val<A>(a) + val<B>(b);
}
template <int A, class R> __device__ __forceinline__ R neg(const R& a) {
  if constexpr (A == kZero) return a;
  else return -val<A>(a);
}
template <int A, int B, class R> __device__ __forceinline__ R sub(const R& a, const R& b) {
  if constexpr (B == kZero) return a;
  else if constexpr (A == kZero) return neg<B>(b);
  else return val<A>(a) - val<B>(b);
}
// a c for a tangent a of kind A and a number c (kind scale_kind(A)).
template <int A, class R> __device__ __forceinline__ R scale(const R& a, const R& c) {
  if constexpr (A == kZero) return a;
  else if constexpr (A == kOne) return c;
  else return a * c;
}
// Product rule: at bv + av bt for tangents at, bt of kinds A, B.
template <int A, int B> __host__ __device__ constexpr int prod_kind() { return add_kind(scale_kind(A), scale_kind(B)); }
template <int A, int B, class R>
__device__ __forceinline__ R prod(const R& at, const R& bv, const R& av, const R& bt) {
  return add<scale_kind(A), scale_kind(B)>(scale<A>(at, bv), scale<B>(bt, av));
}
// Quotient rule with v = a / b, ib = 1 / b: (at - v bt) ib.
template <int A, int B> __host__ __device__ constexpr int quot_kind() { return scale_kind(sub_kind(A, scale_kind(B))); }
template <int A, int B, class R>
__device__ __forceinline__ R quot(const R& at, const R& bt, const R& v, const R& ib) {
  return scale<sub_kind(A, scale_kind(B))>(sub<A, scale_kind(B)>(at, scale<B>(bt, v)), ib);
}
}  // namespace dual

template <class R, int A, int B, int C, int E>
__device__ __forceinline__ D2<R, dual::add_kind(A, C), dual::add_kind(B, E)> operator+(const D2<R, A, B>& a,
                                                                                      const D2<R, C, E>& b) {
  return {a.v + b.v, dual::add<A, C>(a.dr, b.dr), dual::add<B, E>(a.de, b.de)};
}
template <class R, int A, int B, int C, int E>
__device__ __forceinline__ D2<R, dual::sub_kind(A, C), dual::sub_kind(B, E)> operator-(const D2<R, A, B>& a,
                                                                                      const D2<R, C, E>& b) {
  return {a.v - b.v, dual::sub<A, C>(a.dr, b.dr), dual::sub<B, E>(a.de, b.de)};
}
template <class R, int A, int B>
__device__ __forceinline__ D2<R, dual::neg_kind(A), dual::neg_kind(B)> operator-(const D2<R, A, B>& a) {
  return {-a.v, dual::neg<A>(a.dr), dual::neg<B>(a.de)};
}
template <class R, int A, int B, int C, int E>
__device__ __forceinline__ D2<R, dual::prod_kind<A, C>(), dual::prod_kind<B, E>()> operator*(const D2<R, A, B>& a,
                                                                                            const D2<R, C, E>& b) {
  return {a.v * b.v, dual::prod<A, C>(a.dr, b.v, a.v, b.dr), dual::prod<B, E>(a.de, b.v, a.v, b.de)};
}
// Quotient with one reciprocal: v = a/b, dv = (da - v db) / b.
template <class R, int A, int B, int C, int E>
__device__ __forceinline__ D2<R, dual::quot_kind<A, C>(), dual::quot_kind<B, E>()> operator/(const D2<R, A, B>& a,
                                                                                            const D2<R, C, E>& b) {
  const R ib = rcp_(b.v);
  const R v = a.v * ib;
  return {v, dual::quot<A, C>(a.dr, b.dr, v, ib), dual::quot<B, E>(a.de, b.de, v, ib)};
}
// Mixed with numbers of the compute type.
template <class R, int A, int B> __device__ __forceinline__ D2<R, A, B> operator+(const D2<R, A, B>& a, R c) {
  return {a.v + c, a.dr, a.de};
}
template <class R, int A, int B> __device__ __forceinline__ D2<R, A, B> operator+(R c, const D2<R, A, B>& a) {
  return {c + a.v, a.dr, a.de};
}
template <class R, int A, int B> __device__ __forceinline__ D2<R, A, B> operator-(const D2<R, A, B>& a, R c) {
  return {a.v - c, a.dr, a.de};
}
template <class R, int A, int B>
__device__ __forceinline__ D2<R, dual::neg_kind(A), dual::neg_kind(B)> operator-(R c, const D2<R, A, B>& a) {
  return {c - a.v, dual::neg<A>(a.dr), dual::neg<B>(a.de)};
}
template <class R, int A, int B>
__device__ __forceinline__ D2<R, dual::scale_kind(A), dual::scale_kind(B)> operator*(const D2<R, A, B>& a, R c) {
  return {a.v * c, dual::scale<A>(a.dr, c), dual::scale<B>(a.de, c)};
}
template <class R, int A, int B>
__device__ __forceinline__ D2<R, dual::scale_kind(A), dual::scale_kind(B)> operator*(R c, const D2<R, A, B>& a) {
  return {c * a.v, dual::scale<A>(a.dr, c), dual::scale<B>(a.de, c)};
}

// Seeds: the first and the second argument of a two-argument function.
template <class R> __device__ __forceinline__ D2<R, kOne, kZero> arg1(R x) { return {x, R(0), R(0)}; }
template <class R> __device__ __forceinline__ D2<R, kZero, kOne> arg2(R x) { return {x, R(0), R(0)}; }
// A result with both tangents as numbers.
template <class R, int A, int B> __device__ __forceinline__ D2<R> tangents(const D2<R, A, B>& a) {
  return {a.v, dual::val<A>(a.dr), dual::val<B>(a.de)};
}

// EOS parameter slots (KArgs::ke / kef), computed on the host in double:
enum EosSlot { kEA1 = 0, kEIA1, kEB, kEICV, kEPINF, kEQ, kEGP, kEA };
//   gamma - 1, 1/(gamma - 1), b, 1/c_v, p_inf, q, gamma p_inf, a

// Noble-Abel stiffened gas (O. Le Metayer and R. Saurel, Phys. Fluids 28,
// 046102, 2016): p = (gamma-1)(e - q) rho / (1 - b rho) - gamma p_inf,
// T = (e - q - p_inf (1/rho - b)) / c_v.  The ideal gas for p_inf = b = q = 0,
// the stiffened gas for b = 0.
template <class R> struct EosNasg {
  static constexpr bool kIdeal = false;
  R a1, ia1, b, icv, pinf, q, gp;
  template <class X, class Y> __device__ __forceinline__ auto p_rhoe(const X& rho, const Y& e) const {
    return a1 * (e - q) * rho / (R(1) - b * rho) - gp;
  }
  __device__ __forceinline__ R T_rhoe(R rho, R e) const { return (e - q - pinf * (R(1) / rho - b)) * icv; }
  template <class X, class Y> __device__ __forceinline__ auto rhoe_rhop(const X& rho, const Y& p) const {
    return (p + gp) * (R(1) - b * rho) * ia1 + rho * q;
  }
};

// Van der Waals gas with caloric law e = c_v T - a rho:
// p = (gamma-1)(rho e + a rho^2)/(1 - b rho) - a rho^2, T = (e + a rho) / c_v.
template <class R> struct EosVdw {
  static constexpr bool kIdeal = false;
  R a1, ia1, b, icv, a;
  template <class X, class Y> __device__ __forceinline__ auto p_rhoe(const X& rho, const Y& e) const {
    const auto ar2 = a * rho * rho;
    return a1 * (rho * e + ar2) / (R(1) - b * rho) - ar2;
  }
  __device__ __forceinline__ R T_rhoe(R rho, R e) const { return (e + a * rho) * icv; }
  template <class X, class Y> __device__ __forceinline__ auto rhoe_rhop(const X& rho, const Y& p) const {
    const auto ar2 = a * rho * rho;
    return (p + ar2) * (R(1) - b * rho) * ia1 - ar2;
  }
};

// Parameter slot k of the EOS block in compute type R.
template <class R> __device__ __forceinline__ R eos_param(const KArgs& a, int k);
template <> __device__ __forceinline__ double eos_param<double>(const KArgs& a, int k) { return a.ke[k]; }
template <> __device__ __forceinline__ float eos_param<float>(const KArgs& a, int k) { return a.kef[k]; }
template <> __device__ __forceinline__ dw eos_param<dw>(const KArgs& a, int k) { return dw(a.kef[k], a.kel[k]); }

// Model tags: the per-point model type for compute type R and its
// construction from the kernel's parameter block.
struct NasgModel {
  template <class R> using K = EosNasg<R>;
  template <class R> static __device__ __forceinline__ EosNasg<R> make(const KArgs& a) {
    return {eos_param<R>(a, kEA1), eos_param<R>(a, kEIA1), eos_param<R>(a, kEB), eos_param<R>(a, kEICV),
            eos_param<R>(a, kEPINF), eos_param<R>(a, kEQ), eos_param<R>(a, kEGP)};
  }
};
struct VdwModel {
  template <class R> using K = EosVdw<R>;
  template <class R> static __device__ __forceinline__ EosVdw<R> make(const KArgs& a) {
    return {eos_param<R>(a, kEA1), eos_param<R>(a, kEIA1), eos_param<R>(a, kEB), eos_param<R>(a, kEICV),
            eos_param<R>(a, kEA)};
  }
};

}  // namespace fdbb
