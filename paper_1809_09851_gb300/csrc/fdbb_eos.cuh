// fdbb_eos.cuh -- general equations of state for the building-block kernels.
//
// The paper lets a user plug in an equation of state of the form f(p, V, T) = 0
// by writing a type with static members p_rhoe(rho, e) and T_rhoe(rho, e)
// (section 2.2, "Equations of state", Fig. 10).  Here an EOS model is a small
// device struct with the same members plus the inverse rhoe_rhop(rho, p):
//
//   template <class X> X p_rhoe(const X& rho, const X& e) const;   // pressure
//   R T_rhoe(R rho, R e) const;                                     // temperature
//   template <class X> X rhoe_rhop(const X& rho, const X& p) const; // rho e
//
// p_rhoe and rhoe_rhop are templates over the number type X so that the
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
template <class R> struct D2 {
  R v, dr, de;
};

template <class R> __device__ __forceinline__ D2<R> operator+(const D2<R>& a, const D2<R>& b) {
  return {a.v + b.v, a.dr + b.dr, a.de + b.de};
}
template <class R> __device__ __forceinline__ D2<R> operator-(const D2<R>& a, const D2<R>& b) {
  return {a.v - b.v, a.dr - b.dr, a.de - b.de};
}
template <class R> __device__ __forceinline__ D2<R> operator-(const D2<R>& a) { return {-a.v, -a.dr, -a.de}; }
template <class R> __device__ __forceinline__ D2<R> operator*(const D2<R>& a, const D2<R>& b) {
  return {a.v * b.v, a.dr * b.v + a.v * b.dr, a.de * b.v + a.v * b.de};
}
// Quotient with one reciprocal: v = a/b, dv = (da - v db) / b.
template <class R> __device__ __forceinline__ D2<R> operator/(const D2<R>& a, const D2<R>& b) {
  const R ib = rcp_(b.v);
  const R v = a.v * ib;
  return {v, (a.dr - v * b.dr) * ib, (a.de - v * b.de) * ib};
}
// Mixed with constants of the compute type.
template <class R> __device__ __forceinline__ D2<R> operator+(const D2<R>& a, R c) { return {a.v + c, a.dr, a.de}; }
template <class R> __device__ __forceinline__ D2<R> operator+(R c, const D2<R>& a) { return {c + a.v, a.dr, a.de}; }
template <class R> __device__ __forceinline__ D2<R> operator-(const D2<R>& a, R c) { return {a.v - c, a.dr, a.de}; }
template <class R> __device__ __forceinline__ D2<R> operator-(R c, const D2<R>& a) { return {c - a.v, -a.dr, -a.de}; }
template <class R> __device__ __forceinline__ D2<R> operator*(const D2<R>& a, R c) {
  return {a.v * c, a.dr * c, a.de * c};
}
template <class R> __device__ __forceinline__ D2<R> operator*(R c, const D2<R>& a) {
  return {c * a.v, c * a.dr, c * a.de};
}

// Seeds: the first and the second argument of a two-argument function.
template <class R> __device__ __forceinline__ D2<R> arg1(R x) { return {x, R(1), R(0)}; }
template <class R> __device__ __forceinline__ D2<R> arg2(R x) { return {x, R(0), R(1)}; }

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
  template <class X> __device__ __forceinline__ X p_rhoe(const X& rho, const X& e) const {
    return a1 * (e - q) * rho / (R(1) - b * rho) - gp;
  }
  __device__ __forceinline__ R T_rhoe(R rho, R e) const { return (e - q - pinf * (R(1) / rho - b)) * icv; }
  template <class X> __device__ __forceinline__ X rhoe_rhop(const X& rho, const X& p) const {
    return (p + gp) * (R(1) - b * rho) * ia1 + rho * q;
  }
};

// Van der Waals gas with caloric law e = c_v T - a rho:
// p = (gamma-1)(rho e + a rho^2)/(1 - b rho) - a rho^2, T = (e + a rho) / c_v.
template <class R> struct EosVdw {
  static constexpr bool kIdeal = false;
  R a1, ia1, b, icv, a;
  template <class X> __device__ __forceinline__ X p_rhoe(const X& rho, const X& e) const {
    const X ar2 = a * rho * rho;
    return a1 * (rho * e + ar2) / (R(1) - b * rho) - ar2;
  }
  __device__ __forceinline__ R T_rhoe(R rho, R e) const { return (e + a * rho) * icv; }
  template <class X> __device__ __forceinline__ X rhoe_rhop(const X& rho, const X& p) const {
    const X ar2 = a * rho * rho;
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
