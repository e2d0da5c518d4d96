// fdbb_kernels.cuh -- one fused kernel per building block.
//
// Each block evaluates one expression tree point by point: Op::apply takes the
// input planes of VW consecutive points (storage type T) from a *source*,
// converts them to the compute type R, evaluates the expressions in registers
// and stores every output plane once.  No temporaries touch memory.
//
// Two kernels drive the ops:
//   k_pointwise -- a persistent grid strides over chunks of VW points and
//                  reads them straight from global memory (GlobalSrc);
//   k_staged    -- a persistent grid walks 256*VW-point tiles; one thread per
//                  block streams the input planes of the block's next tiles
//                  into a two-stage shared-memory ring with bulk asynchronous
//                  copies (cp.async.bulk, completion on an mbarrier) while the
//                  block computes the current tile from the other stage
//                  (SmemSrc), so HBM latency overlaps the arithmetic.  The
//                  ragged tail (< one tile) is read straight from global
//                  memory.
//
// apply() returns false -- before storing anything -- when the double-word
// range guard fails; the chunk is then recomputed in native FP64 from the same
// source.
#pragma once

#include <atomic>
#include <type_traits>

#include "fdbb_device.cuh"
#include "fdbb_internal.h"

namespace fdbb {

constexpr int kThreads = 256;
constexpr int kStages = 2;
constexpr int kWaitLimit = 1 << 22;  // bounded mbarrier polls per wait

template <class T> __device__ __forceinline__ const T* inp(const KArgs& a, int k) {
  return static_cast<const T*>(a.in[k]);
}
template <class T> __device__ __forceinline__ T* outp(const KArgs& a, int k) {
  return static_cast<T*>(a.out[k]);
}

template <class R> __device__ __forceinline__ Consts<R> consts(const KArgs& a);
template <> __device__ __forceinline__ Consts<double> consts<double>(const KArgs& a) {
  return {a.kd[0], a.kd[1], a.kd[2], a.kd[3], a.kd[4], a.kd[5], a.kd[6], a.kd[7]};
}
template <> __device__ __forceinline__ Consts<float> consts<float>(const KArgs& a) {
  return {a.kf[0], a.kf[1], a.kf[2], a.kf[3], a.kf[4], a.kf[5], a.kf[6], a.kf[7]};
}
template <> __device__ __forceinline__ Consts<dw> consts<dw>(const KArgs& a) {
  return {dw(a.kf[0], a.kl[0]), dw(a.kf[1], a.kl[1]), dw(a.kf[2], a.kl[2]), dw(a.kf[3], a.kl[3]),
          dw(a.kf[4], a.kl[4]), dw(a.kf[5], a.kl[5]), dw(a.kf[6], a.kl[6]), dw(a.kf[7], a.kl[7])};
}
// The float constants in both lanes of packed float pairs.
__device__ __forceinline__ Consts<fl2> splat_consts(const Consts<float>& k) {
  return {fl2(k.g), fl2(k.a1), fl2(k.g3), fl2(k.ta1), fl2(k.ia1), fl2(k.mg), fl2(k.gia1), fl2(k.tcv)};
}
// The double-word constants in both lanes of packed values.
__device__ __forceinline__ Consts<dw2> splat_consts(const Consts<dw>& k) {
  return {splat2(k.g), splat2(k.a1), splat2(k.g3), splat2(k.ta1),
          splat2(k.ia1), splat2(k.mg), splat2(k.gia1), splat2(k.tcv)};
}

// Model tag of the ideal gas (the general-EOS tags are in fdbb_eos.cuh).
struct IdealModel {
  template <class R> static __device__ __forceinline__ Consts<R> make(const KArgs& a) { return consts<R>(a); }
};

// ---------------------------------------------------------------------------
// Input sources: plane k of the current VW points, in the storage's load type.
// ---------------------------------------------------------------------------

// Straight from global memory (cnt < VW only in the ragged last chunk).
template <class T, int VW> struct GlobalSrc {
  static constexpr DwConv kConv = DwConv::kClamp;
  const KArgs& a;
  int64_t i0;
  int cnt;
  __device__ __forceinline__ void raw(int k, typename Storage<T>::L (&r)[VW], float fill) const {
    if (!FDBB_IDX_OK(a.dbg, k >= 0 && k < a.nin && i0 >= 0 && cnt >= 1 && cnt <= VW && i0 + cnt <= a.n, i0)) {
#pragma unroll
      for (int j = 0; j < VW; ++j) r[j] = static_cast<typename Storage<T>::L>(fill);
      return;
    }
    load_raw<T, VW>(inp<T>(a, k), i0, cnt, r, fill);
  }
};

// From the block's shared-memory stage: this thread's VW points of plane k sit
// at base + k * TILE (the stage stays valid until the block has finished the
// tile, so a double-word chunk can be re-read for its FP64 fallback).
template <class T, int VW, int TILE> struct SmemSrc {
  static constexpr DwConv kConv = DwConv::kClamp;
  const T* base;
#ifdef FDBB_DEBUG
  int nin;  // planes staged in the ring
  unsigned long long* dbg;
#endif
  __device__ __forceinline__ void raw(int k, typename Storage<T>::L (&r)[VW], float fill) const {
#ifdef FDBB_DEBUG
    if (!FDBB_IDX_OK(dbg, k >= 0 && k < nin, k)) {
#pragma unroll
      for (int j = 0; j < VW; ++j) r[j] = static_cast<typename Storage<T>::L>(fill);
      return;
    }
#endif
    ld_sh(base + (size_t)k * TILE, r);
  }
};

// Output plane k of the current VW points (a NULL plane is skipped), in the
// source's conversion form.
// (cnt counts points: up to VW, or 2 for one packed pair of points.)
template <class T, int VW, class R, class Src>
__device__ __forceinline__ void put(const KArgs& a, const Src&, int k, int64_t i0, int cnt, const R (&x)[VW]) {
  if (!FDBB_IDX_OK(a.dbg, k >= 0 && k < kMaxOut && i0 >= 0 && cnt >= 1 && i0 + cnt <= a.n, i0)) return;
  store_c<T, VW, R, Src::kConv>(outp<T>(a, k), i0, cnt, x);
}
template <class T, int VW, class Src, class L>
__device__ __forceinline__ void put_raw(const KArgs& a, const Src&, int k, int64_t i0, int cnt, const L (&raw)[VW]) {
  if (!FDBB_IDX_OK(a.dbg, k >= 0 && k < kMaxOut && i0 >= 0 && cnt >= 1 && i0 + cnt <= a.n, i0)) return;
  store_raw<T, VW>(outp<T>(a, k), i0, cnt, raw);
}

// Conservative state of VW points from input planes base..base+D+1.
template <class T, int VW, int D, class R, class G, class Src>
__device__ __forceinline__ void load_U(const Src& src, int base, Pt<R, D> (&s)[VW], G& g) {
  typename LoadOf<T, R>::type raw[VW];
  src.raw(base, raw, 1.0f);
#pragma unroll
  for (int j = 0; j < VW; ++j) {
    s[j].rho = to_compute_c<R, Src::kConv>(raw[j], g);
    if constexpr (IsDw<R>::value) s[j].raw.rho = raw[j];
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    src.raw(base + 1 + i, raw, 0.0f);
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      s[j].m[i] = to_compute_c<R, Src::kConv>(raw[j], g);
      if constexpr (IsDw<R>::value) s[j].raw.m[i] = raw[j];
    }
  }
  src.raw(base + D + 1, raw, 1.0f);
#pragma unroll
  for (int j = 0; j < VW; ++j) s[j].rE = to_compute_c<R, Src::kConv>(raw[j], g);
}

// One plane, converted to the compute type.
template <class T, int VW, class R, class G, class Src>
__device__ __forceinline__ void load_plane(const Src& src, int k, R (&x)[VW], float fill, G& g) {
  typename LoadOf<T, R>::type raw[VW];
  src.raw(k, raw, fill);
#pragma unroll
  for (int j = 0; j < VW; ++j) x[j] = to_compute_c<R, Src::kConv>(raw[j], g);
}

// nv planes of a second input field (W or G) from planes base..base+nv-1,
// as w[point][component].
template <class T, int VW, int NV, class R, class G, class Src>
__device__ __forceinline__ void load_field(const Src& src, int base, R (&w)[VW][NV], G& g) {
  R x[VW];
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    load_plane<T, VW, R>(src, base + c, x, 0.0f, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) w[j][c] = x[j];
  }
}

// Sums of storage words, lane by lane for pairs.
__device__ __forceinline__ double ladd(double x, double y) { return x + y; }
__device__ __forceinline__ float ladd(float x, float y) { return x + y; }
__device__ __forceinline__ double2 ladd(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }
__device__ __forceinline__ double lsub(double x, double y) { return x - y; }
__device__ __forceinline__ float lsub(float x, float y) { return x - y; }
__device__ __forceinline__ double2 lsub(double2 x, double2 y) { return make_double2(x.x - y.x, x.y - y.y); }
__device__ __forceinline__ float2 ladd(float2 x, float2 y) { return make_float2(x.x + y.x, x.y + y.y); }
__device__ __forceinline__ float2 lsub(float2 x, float2 y) { return make_float2(x.x - y.x, x.y - y.y); }

// Characteristic weights W (planes base..base+NV-1, inputs) for the inverse
// transform, with the three sums of weights it needs -- w_1 + w_2 + w_nv,
// w_nv - w_1 and w_1 + w_nv -- formed in the storage's own IEEE type before
// the conversion to R: sums of two exact inputs can cancel, and a double-word
// value carries ~47 of a double's 53 bits, so in double-word arithmetic they
// would not be accurate relative to their own magnitude.
template <class T, int VW, int NV, class R, class G, class Src>
__device__ __forceinline__ void load_weights_inv(const Src& src, int base, R (&w)[VW][NV], R (&sum)[VW],
                                                 R (&anm1)[VW], R (&a1pn)[VW], G& g) {
  using L = typename LoadOf<T, R>::type;
  L raw[NV][VW];
#pragma unroll
  for (int c = 0; c < NV; ++c) src.raw(base + c, raw[c], 0.0f);
#pragma unroll
  for (int j = 0; j < VW; ++j) {
#pragma unroll
    for (int c = 0; c < NV; ++c) w[j][c] = to_compute_c<R, Src::kConv>(raw[c][j], g);
    const L a1 = raw[0][j], a2 = raw[1][j], an = raw[NV - 1][j];
    sum[j] = to_compute_c<R, Src::kConv>(ladd(ladd(a1, a2), an), g);
    anm1[j] = to_compute_c<R, Src::kConv>(lsub(an, a1), g);
    a1pn[j] = to_compute_c<R, Src::kConv>(ladd(a1, an), g);
  }
}

// Store y[point][component] into output planes base..base+NV-1.
template <class T, int VW, int NV, class R, class Src>
__device__ __forceinline__ void store_field(const KArgs& a, const Src& src, int base, int64_t i0, int cnt,
                                            const R (&y)[VW][NV]) {
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    if (!outp<T>(a, base + c)) continue;
    R x[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) x[j] = y[j][c];
    put<T, VW, R>(a, src, base + c, i0, cnt, x);
  }
}

template <int VW, int D, bool C2 = true, bool WH = true, bool WQ = WH, class R, class K, class G>
__device__ __forceinline__ void derive_all(Pt<R, D> (&s)[VW], const K& k, G& g) {
#pragma unroll
  for (int j = 0; j < VW; ++j) derive<C2, WH, WQ>(s[j], k, g);
}

// Flux column d into output planes base..base+nv-1.  Component 0 is the input
// momentum m_d itself, stored bit for bit.
template <class T, int VW, int D, int d, class R, class Src>
__device__ __forceinline__ void emit_flux(const KArgs& a, const Src& src, int base, int64_t i0, int cnt,
                                          const Pt<R, D> (&s)[VW]) {
#pragma unroll
  for (int c = 0; c < D + 2; ++c) {
    if (!outp<T>(a, base + c)) continue;
    if constexpr (IsDw<R>::value) {
      if (c == 0) {  // F_d[0] = m_d: the input itself, bit for bit
        typename LoadOf<T, R>::type raw[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) raw[j] = s[j].raw.m[d];
        put_raw<T, VW>(a, src, base + c, i0, cnt, raw);
        continue;
      }
    }
    R x[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) x[j] = flux_comp<D, d>(s[j], c);
    put<T, VW, R>(a, src, base + c, i0, cnt, x);
  }
}

// Jacobian A_d into output planes base..base+nv*nv-1 (row-major).
template <class T, int VW, int D, int d, class R, class K, class Src>
__device__ __forceinline__ void emit_jac(const KArgs& a, const Src& src, int base, int64_t i0, int cnt,
                                         const Pt<R, D> (&s)[VW], const K& k) {
  constexpr int nv = D + 2;
#pragma unroll
  for (int row = 0; row < nv; ++row) {
#pragma unroll
    for (int col = 0; col < nv; ++col) {
      if (!outp<T>(a, base + row * nv + col)) continue;
      R x[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) x[j] = jac_entry<D, d>(s[j], k, row, col);
      put<T, VW, R>(a, src, base + row * nv + col, i0, cnt, x);
    }
  }
}

// ---------------------------------------------------------------------------
// Ops.  kIn = number of input planes; apply<T, VW, R>(a, k, src, i0, cnt).
// ---------------------------------------------------------------------------

// |v|^2 = (sum m_i^2) / (rho rho)  (paper section 3, Eq. (2)).
template <int D> struct OpVMag2 {
  static constexpr int kIn = D + 1;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K&, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    R rho[VW], m[VW], num[VW];
    load_plane<T, VW, R>(src, 0, rho, 1.0f, g);
    load_plane<T, VW, R>(src, 1, m, 0.0f, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) num[j] = m[j] * m[j];
#pragma unroll
    for (int i = 1; i < D; ++i) {
      load_plane<T, VW, R>(src, 1 + i, m, 0.0f, g);
#pragma unroll
      for (int j = 0; j < VW; ++j) num[j] = fma_(m[j], m[j], num[j]);
    }
    if (!g.ok) return false;
#pragma unroll
    for (int j = 0; j < VW; ++j) num[j] = num[j] / (rho[j] * rho[j]);
    store<T, VW, R>(outp<T>(a, 0), i0, cnt, num);
    return true;
  }
};

// V = (rho, v, p) from U.
template <int D> struct OpPrim {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    derive_all<VW, D, false>(s, k, g);
    if (!g.ok) return false;
    R x[VW];
    if constexpr (IsDw<R>::value) {
      typename LoadOf<T, R>::type raw[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) raw[j] = s[j].raw.rho;
      store_raw<T, VW>(outp<T>(a, 0), i0, cnt, raw);
    } else {
#pragma unroll
      for (int j = 0; j < VW; ++j) x[j] = s[j].rho;
      store<T, VW, R>(outp<T>(a, 0), i0, cnt, x);
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
      for (int j = 0; j < VW; ++j) x[j] = s[j].v[i];
      store<T, VW, R>(outp<T>(a, 1 + i), i0, cnt, x);
    }
#pragma unroll
    for (int j = 0; j < VW; ++j) x[j] = s[j].p;
    store<T, VW, R>(outp<T>(a, D + 1), i0, cnt, x);
    return true;
  }
};

// U = (rho, rho v, p/(gamma-1) + rho |v|^2 / 2) from V; for a general EOS
// rhoE = rho e(rho, p) + rho |v|^2 / 2.
template <int D> struct OpCons {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    R rho[VW], v[D][VW], p[VW], x[VW];
    typename LoadOf<T, R>::type rho_raw[VW];
    src.raw(0, rho_raw, 1.0f);
#pragma unroll
    for (int j = 0; j < VW; ++j) rho[j] = to_compute_c<R, Src::kConv>(rho_raw[j], g);
#pragma unroll
    for (int i = 0; i < D; ++i) load_plane<T, VW, R>(src, 1 + i, v[i], 0.0f, g);
    load_plane<T, VW, R>(src, D + 1, p, 1.0f, g);
    if (!g.ok) return false;
    store_raw<T, VW>(outp<T>(a, 0), i0, cnt, rho_raw);  // rho: a copy of the input
    R v2[VW];
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
      for (int j = 0; j < VW; ++j) {
        v2[j] = (i == 0) ? v[i][j] * v[i][j] : fma_(v[i][j], v[i][j], v2[j]);
        x[j] = rho[j] * v[i][j];
      }
      store<T, VW, R>(outp<T>(a, 1 + i), i0, cnt, x);
    }
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      if constexpr (K::kIdeal)
        x[j] = fma_(p[j], k.ia1, half_(rho[j] * v2[j]));
      else
        x[j] = k.rhoe_rhop(rho[j], p[j]) + half_(rho[j] * v2[j]);
    }
    store<T, VW, R>(outp<T>(a, D + 1), i0, cnt, x);
    return true;
  }
};

// p and c.
template <int D> struct OpEos {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    derive_all<VW, D, true, false>(s, k, g);
    if (!g.ok) return false;
    R x[VW];
    if (T* o = outp<T>(a, 0)) {
#pragma unroll
      for (int j = 0; j < VW; ++j) x[j] = s[j].p;
      store<T, VW, R>(o, i0, cnt, x);
    }
    if (T* o = outp<T>(a, 1)) {
#pragma unroll
      for (int j = 0; j < VW; ++j) x[j] = sqrt_(s[j].c2);
      store<T, VW, R>(o, i0, cnt, x);
    }
    return true;
  }
};

// w- = u - 2c/(gamma-1), w+ = u + 2c/(gamma-1), s = p rho^-gamma.
template <int D, int d> struct OpRiemann {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    derive_all<VW, D, true, false>(s, k, g);
    if (!g.ok) return false;
    R wm[VW], wp[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      const R tc = k.ta1 * sqrt_(s[j].c2);
      wm[j] = s[j].v[d] - tc;
      wp[j] = s[j].v[d] + tc;
    }
    store<T, VW, R>(outp<T>(a, 0), i0, cnt, wm);
    store<T, VW, R>(outp<T>(a, 1), i0, cnt, wp);
    if (T* o = outp<T>(a, 2)) {
#pragma unroll
      for (int j = 0; j < VW; ++j) wm[j] = s[j].p * pow_(s[j].rho, k.mg);
      store<T, VW, R>(o, i0, cnt, wm);
    }
    return true;
  }
};

// Flux column d, or all columns when d == -1.
template <int D, int d> struct OpFlux {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    derive_all<VW, D, false, false>(s, k, g);
    if (!g.ok) return false;
    if constexpr (d >= 0) {
      emit_flux<T, VW, D, d>(a, src, 0, i0, cnt, s);
    } else {
      emit_flux<T, VW, D, 0>(a, src, 0, i0, cnt, s);
      if constexpr (D > 1) emit_flux<T, VW, D, 1>(a, src, D + 2, i0, cnt, s);
      if constexpr (D > 2) emit_flux<T, VW, D, 2>(a, src, 2 * (D + 2), i0, cnt, s);
    }
    return true;
  }
};

template <int D, int d> struct OpJac {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    derive_all<VW, D, false>(s, k, g);
    if (!g.ok) return false;
    emit_jac<T, VW, D, d>(a, src, 0, i0, cnt, s, k);
    return true;
  }
};

template <int D, int d, bool INV> struct OpChar {
  static constexpr int kIn = 2 * (D + 2);
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    R w[VW][nv], y[VW][nv];
    if constexpr (INV) {
      R sum[VW], anm1[VW], a1pn[VW];
      load_weights_inv<T, VW, nv>(src, nv, w, sum, anm1, a1pn, g);
      derive_all<VW, D>(s, k, g);
      if (!g.ok) return false;
#pragma unroll
      for (int j = 0; j < VW; ++j) char_inv_sums<D, d>(s[j], k, w[j], sum[j], anm1[j], a1pn[j], y[j]);
    } else {
      load_field<T, VW, nv>(src, nv, w, g);
      derive_all<VW, D, true, false, true>(s, k, g);
      if (!g.ok) return false;
#pragma unroll
      for (int j = 0; j < VW; ++j) char_fwd<D, d>(s[j], k, w[j], y[j]);
    }
    store_field<T, VW, nv>(a, src, 0, i0, cnt, y);
    return true;
  }
};

template <int D, int d> using OpCharFwd = OpChar<D, d, false>;
template <int D, int d> using OpCharInv = OpChar<D, d, true>;

// All flux columns (planes 0..D*nv-1), A_dj (D*nv .. D*nv+nv^2-1) and
// L_dj W (last nv planes) in one pass; inputs U (planes 0..nv-1), W (nv..2nv-1).
template <int D, int dj> struct OpFused {
  static constexpr int kIn = 2 * (D + 2);
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    R w[VW][nv];
    const bool want_y = a.in[nv] != nullptr;
    if (want_y) load_field<T, VW, nv>(src, nv, w, g);
    derive_all<VW, D>(s, k, g);
    if (!g.ok) return false;
    emit_flux<T, VW, D, 0>(a, src, 0, i0, cnt, s);
    if constexpr (D > 1) emit_flux<T, VW, D, 1>(a, src, nv, i0, cnt, s);
    if constexpr (D > 2) emit_flux<T, VW, D, 2>(a, src, 2 * nv, i0, cnt, s);
    emit_jac<T, VW, D, dj>(a, src, D * nv, i0, cnt, s, k);
    if (want_y) {
      R y[VW][nv];
#pragma unroll
      for (int j = 0; j < VW; ++j) char_fwd<D, dj>(s[j], k, w[j], y[j]);
      store_field<T, VW, nv>(a, src, D * nv + nv * nv, i0, cnt, y);
    }
    return true;
  }
};

template <int D, int d> struct OpVjp {
  static constexpr int kIn = 2 * (D + 2);
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    R gg[VW][nv], y[VW][nv];
    load_field<T, VW, nv>(src, nv, gg, g);
    derive_all<VW, D, false>(s, k, g);
    if (!g.ok) return false;
#pragma unroll
    for (int j = 0; j < VW; ++j) flux_vjp_pt<D, d>(s[j], k, gg[j], y[j]);
    store_field<T, VW, nv>(a, src, 0, i0, cnt, y);
    return true;
  }
};

// Roe flux between U_L (planes 0..nv-1) and U_R (nv..2nv-1) in direction d.
template <int D, int d> struct OpRoeFlux {
  static constexpr int kIn = 2 * (D + 2);
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> L[VW], Rt[VW], s[VW];
    load_U<T, VW, D>(src, 0, L, g);
    load_U<T, VW, D>(src, nv, Rt, g);
    derive_all<VW, D, false, true, false>(L, k, g);
    derive_all<VW, D, false, true, false>(Rt, k, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) roe_state(L[j], Rt[j], k, s[j], g);
    if (!g.ok) return false;
    R y[VW][nv];
#pragma unroll
    for (int j = 0; j < VW; ++j) roe_flux_pt<D, d>(L[j], Rt[j], s[j], k, y[j]);
    store_field<T, VW, nv>(a, src, 0, i0, cnt, y);
    return true;
  }
};

// Characteristic transform at the Roe-averaged state of U_L (planes 0..nv-1)
// and U_R (nv..2nv-1) applied to W (2nv..3nv-1).
template <int D, int d, bool INV> struct OpRoeChar {
  static constexpr int kIn = 3 * (D + 2);
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> L[VW], Rt[VW], s[VW];
    load_U<T, VW, D>(src, 0, L, g);
    load_U<T, VW, D>(src, nv, Rt, g);
    R w[VW][nv], y[VW][nv];
    R sum[VW], anm1[VW], a1pn[VW];
    if constexpr (INV)
      load_weights_inv<T, VW, nv>(src, 2 * nv, w, sum, anm1, a1pn, g);
    else
      load_field<T, VW, nv>(src, 2 * nv, w, g);
    derive_all<VW, D, false, true, false>(L, k, g);
    derive_all<VW, D, false, true, false>(Rt, k, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) roe_state(L[j], Rt[j], k, s[j], g);
    if (!g.ok) return false;
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      if constexpr (INV)
        char_inv_sums<D, d>(s[j], k, w[j], sum[j], anm1[j], a1pn[j], y[j]);
      else
        char_fwd<D, d>(s[j], k, w[j], y[j]);
    }
    store_field<T, VW, nv>(a, src, 0, i0, cnt, y);
    return true;
  }
};

// Primitive state (rho, v, p) of VW points from planes base..base+D+1; for
// double-word the loaded doubles of rho and v stay available (raw.rho,
// raw.m[i]) for outputs that are copies of them.
template <class T, int VW, int D, class R, class G, class Src>
__device__ __forceinline__ void load_V(const Src& src, int base, Pt<R, D> (&s)[VW], G& g) {
  typename LoadOf<T, R>::type raw[VW];
  src.raw(base, raw, 1.0f);
#pragma unroll
  for (int j = 0; j < VW; ++j) {
    s[j].rho = to_compute_c<R, Src::kConv>(raw[j], g);
    if constexpr (IsDw<R>::value) s[j].raw.rho = raw[j];
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    src.raw(base + 1 + i, raw, 0.0f);
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      s[j].v[i] = to_compute_c<R, Src::kConv>(raw[j], g);
      if constexpr (IsDw<R>::value) s[j].raw.m[i] = raw[j];
    }
  }
  src.raw(base + D + 1, raw, 1.0f);
#pragma unroll
  for (int j = 0; j < VW; ++j) s[j].p = to_compute_c<R, Src::kConv>(raw[j], g);
}

// Inviscid flux from primitive variables V (planes 0..nv-1): column d, or
// all columns when d == -1 (paper section 2.2, Figs. 9 and 11).
template <int D, int d> struct OpFluxPrim {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_V<T, VW, D>(src, 0, s, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) derive_prim(s[j], k, g);
    if (!g.ok) return false;
    constexpr int dlo = d >= 0 ? d : 0, dhi = d >= 0 ? d : D - 1;
#pragma unroll
    for (int dd = dlo; dd <= dhi; ++dd) {
      const int base = d >= 0 ? 0 : dd * (D + 2);
#pragma unroll
      for (int c = 0; c < D + 2; ++c) {
        T* o = outp<T>(a, base + c);
        if (!o) continue;
        R x[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) {
          if (dd == 0) x[j] = flux_comp<D, 0>(s[j], c);
          if constexpr (D > 1) if (dd == 1) x[j] = flux_comp<D, (D > 1 ? 1 : 0)>(s[j], c);
          if constexpr (D > 2) if (dd == 2) x[j] = flux_comp<D, (D > 2 ? 2 : 0)>(s[j], c);
        }
        store<T, VW, R>(o, i0, cnt, x);
      }
    }
    return true;
  }
};

// B_d = dF_d/dV, nv*nv planes row-major.
template <int D, int d> struct OpJacPrim {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_V<T, VW, D>(src, 0, s, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) derive_prim(s[j], k, g);
    if (!g.ok) return false;
#pragma unroll
    for (int row = 0; row < nv; ++row) {
#pragma unroll
      for (int col = 0; col < nv; ++col) {
        T* o = outp<T>(a, row * nv + col);
        if (!o) continue;
        if constexpr (IsDw<R>::value) {
          if (row == 0 && (col == 0 || col == 1 + d)) {  // u and rho: copies of the inputs
            typename LoadOf<T, R>::type raw[VW];
#pragma unroll
            for (int j = 0; j < VW; ++j) raw[j] = col == 0 ? s[j].raw.m[d] : s[j].raw.rho;
            store_raw<T, VW>(o, i0, cnt, raw);
            continue;
          }
        }
        R x[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) x[j] = jacp_entry<D, d>(s[j], k, row, col);
        store<T, VW, R>(o, i0, cnt, x);
      }
    }
    return true;
  }
};

// Temperature T = e / c_v = p / rho / ((gamma - 1) c_v) (paper section 2.2,
// "Equations of state", T_rhoe of the EOS prototype, Fig. 10); a general EOS
// evaluates its own T_rhoe(rho, e).
template <int D> struct OpTemp {
  static constexpr int kIn = D + 2;
  template <class T, int VW, class R, class K, class Src>
  static __device__ __forceinline__ bool apply(const KArgs& a, const K& k, const Src& src, int64_t i0,
                                               int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(src, 0, s, g);
    derive_all<VW, D, false, false>(s, k, g);
    if (!g.ok) return false;
    R x[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      if constexpr (K::kIdeal)
        x[j] = s[j].p * s[j].r * k.tcv;
      else
        x[j] = k.T_rhoe(s[j].rho, s[j].ie);
    }
    store<T, VW, R>(outp<T>(a, 0), i0, cnt, x);
    return true;
  }
};

// ---------------------------------------------------------------------------
// Bulk asynchronous copies and mbarriers (sm_90+ PTX, used on sm_103a)
// ---------------------------------------------------------------------------

// Bounded mbarrier waits that ran out in this translation unit's kernels.
static __device__ unsigned int g_wait_timeouts;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Order this thread's earlier shared-memory accesses before later accesses of
// the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// bytes from global src to shared dst; both 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Wait for the phase with the given parity to complete; false after `limit`
// polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = kWaitLimit) {
  const uint32_t addr = smem_addr(bar);
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Points per thread and plane of an op: the storage's width (one point in
// double-word arithmetic), except the ideal-gas double-word blocks below,
// which take two points per thread -- as two independent scalar double-word
// points (kPairs), or as the two lanes of packed FP32x2 double-word values
// (kPacked, dw2): each FP32 step of the double-word algebra is then one
// FADD2 / FMUL2 / FFMA2 for both points, while the splits and rebuilds of the
// doubles stay per point.  Each lane performs the scalar double-word
// operation's FP32 steps, in the same order and with the same roundings, so a
// point's result does not depend on its partner.  The choice per block is the
// faster one of an A/B at N = 2^26 on one GB300 (fraction of the measured HBM
// bandwidth).  With the select form of the conversions (DwConvOf), one point
// / two points / two points packed:
//   v_mag2 0.79 / 0.94 / 0.98, EOS 0.62 / 0.68 / 0.69, cons -> prim
//   0.77 / 0.87 / 0.89, prim -> cons 0.91 / 0.91 / 0.89, Riemann invariants
//   0.60 / 0.64 / 0.67, one flux column 0.73 / 0.81 / 0.77, all columns
//   0.88 / 0.89 / 0.90, Jacobian 0.86 / 0.88 / 0.88, temperature
//   0.60 / 0.70 / 0.69, all primitive-form columns 0.83 / 0.81 / 0.85,
//   forward characteristic transform 0.66 / - / 0.73, inverse 0.61 / - /
//   0.55, flux VJP - / 0.60 / 0.69; the fused pass 13.35 / - / 13.58
//   Gpoints/s.  With the clamped form, the kept mode against the other
//   candidate: EOS packed 0.82 / two points 0.74, Riemann invariants packed
//   0.75 / two points 0.68, one flux column two points 0.91 / packed 0.89,
//   prim -> cons two points 0.90 / packed 0.90, temperature packed 0.83 /
//   two points 0.77, inverse characteristic transform packed 0.74 / one point
//   0.65.  The Roe-averaged forms need 160-230 registers packed and keep one
//   point.
enum class DwMode { Single, Pairs, Packed };
template <class Op> struct DwModeOf { static constexpr DwMode value = DwMode::Single; };
template <int D> struct DwModeOf<OpVMag2<D>> { static constexpr DwMode value = DwMode::Packed; };
template <int D> struct DwModeOf<OpEos<D>> { static constexpr DwMode value = DwMode::Packed; };
template <int D> struct DwModeOf<OpPrim<D>> { static constexpr DwMode value = DwMode::Packed; };
template <int D> struct DwModeOf<OpCons<D>> { static constexpr DwMode value = DwMode::Pairs; };
template <int D> struct DwModeOf<OpTemp<D>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpRiemann<D, d>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpFlux<D, d>> {
  static constexpr DwMode value = d < 0 ? DwMode::Packed : DwMode::Pairs;
};
template <int D, int d> struct DwModeOf<OpCharInv<D, d>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpFluxPrim<D, d>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpJac<D, d>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpJacPrim<D, d>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpVjp<D, d>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpCharFwd<D, d>> { static constexpr DwMode value = DwMode::Packed; };
template <int D, int d> struct DwModeOf<OpFused<D, d>> { static constexpr DwMode value = DwMode::Packed; };

// Conversion form (fdbb_dw.cuh) of the packed double-word ops: the clamped
// sequences, except for the fused pass, whose 45 outputs hold its kernel at
// the 128-register bound of two blocks per SM and which is faster with the
// selects.  A/B at N = 2^26 on one GB300, clamp / select (fraction of the
// measured HBM bandwidth): EOS 0.82 / 0.69, Riemann invariants 0.75 / 0.67,
// one flux column 0.91 / 0.81, forward characteristic transform 0.83 / 0.73,
// flux VJP 0.78 / 0.69, temperature 0.77 / 0.70, cons -> prim 0.91 / 0.89,
// the rest within 0.03; the fused pass 13.47 / 13.55 Gpoints/s (13.28 /
// 13.38 on a second box).
template <class Op> struct DwConvOf { static constexpr DwConv value = DwConv::kClamp; };
template <int D, int d> struct DwConvOf<OpFused<D, d>> { static constexpr DwConv value = DwConv::kSelect; };

// The float-arithmetic ideal-gas blocks (FP32, FP16, BF16 storage) evaluate a
// thread's four points as two packed FP32x2 pairs (fl2): the same registers,
// about half the FP32 instructions.  A/B at N = 2^26 on one GB300 (fraction of
// the measured HBM bandwidth, scalar / packed; FP32, BF16): EOS 0.91 / 0.95,
// 0.70 / 0.80; Riemann invariants 0.90 / 0.93, 0.66 / 0.76; temperature
// 1.04 / 1.03, 0.70 / 0.78; L.W 0.95 / 0.97, 0.87 / 0.91; flux VJP 0.94 / 0.97,
// 0.90 / 0.91; Roe flux 0.81 / 0.88, 0.42 / 0.46; one flux column 0.92 / 0.93,
// 0.88 / 0.91; the rest within 0.01, except cons -> prim (BF16 0.87 / 0.84) and
// R.W (BF16 0.97 / 0.93), which stay scalar, as does the fused pass (27.6 and
// 55.1 Gpoints/s either way).
template <class Op> struct FloatPacked { static constexpr bool value = true; };
template <int D> struct FloatPacked<OpPrim<D>> { static constexpr bool value = false; };
template <int D, int d> struct FloatPacked<OpCharInv<D, d>> { static constexpr bool value = false; };
template <int D, int d> struct FloatPacked<OpFused<D, d>> { static constexpr bool value = false; };

template <class Op, class T, class R, class Mdl> struct OpWidth {
  static constexpr DwMode kMode = (std::is_same<T, double>::value && std::is_same<R, dw>::value &&
                                   std::is_same<Mdl, IdealModel>::value)
                                      ? DwModeOf<Op>::value
                                      : DwMode::Single;
  static constexpr bool kPacked = kMode == DwMode::Packed;
  static constexpr int VW = kMode == DwMode::Single ? Width<T, R>::VW : 2;
  static constexpr bool kPackedF = FloatPacked<Op>::value && std::is_same<R, float>::value &&
                                   std::is_same<Mdl, IdealModel>::value && VW == 4;
};

// A source of two points per plane presented as one packed value: its storage
// word is the pair of doubles.
template <class Src, DwConv C = DwConv::kClamp> struct PairSrc {
  static constexpr DwConv kConv = C;
  const Src& s;
  __device__ __forceinline__ void raw(int k, double2 (&r)[1], float fill) const {
    double t[2];
    s.raw(k, t, fill);
    r[0] = make_double2(t[0], t[1]);
  }
};

// Four points per plane presented as two packed float pairs: its storage
// words are pairs of floats.
template <class Src> struct QuadSrc {
  static constexpr DwConv kConv = DwConv::kClamp;
  const Src& s;
  __device__ __forceinline__ void raw(int k, float2 (&r)[2], float fill) const {
    float t[4];
    s.raw(k, t, fill);
    r[0] = make_float2(t[0], t[1]);
    r[1] = make_float2(t[2], t[3]);
  }
};

template <class Op, class T, class R, class Mdl, class K, class Src>
__device__ __forceinline__ void apply_chunk(const KArgs& a, const K& k, const Src& src, int64_t i0, int cnt) {
  constexpr int VW = OpWidth<Op, T, R, Mdl>::VW;
  if constexpr (OpWidth<Op, T, R, Mdl>::kPackedF) {
    // float arithmetic on two packed pairs (cnt points, up to four)
    const QuadSrc<Src> qs{src};
    Op::template apply<T, 2, fl2>(a, splat_consts(k), qs, i0, cnt);
  } else if constexpr (OpWidth<Op, T, R, Mdl>::kPacked) {
    // packed double-word fast path (cnt points, 1 or 2); a pair with a value
    // outside its range runs in native FP64
    const PairSrc<Src, DwConvOf<Op>::value> ps{src};
    if (!Op::template apply<T, 1, dw2>(a, splat_consts(k), ps, i0, cnt))
      Op::template apply<T, VW, double>(a, Mdl::template make<double>(a), src, i0, cnt);
  } else if constexpr (std::is_same<R, dw>::value) {
    // double-word fast path; chunks outside its range run in native FP64
    if (!Op::template apply<T, VW, dw>(a, k, src, i0, cnt))
      Op::template apply<T, VW, double>(a, Mdl::template make<double>(a), src, i0, cnt);
  } else {
    Op::template apply<T, VW, R>(a, k, src, i0, cnt);
  }
}

// Chunks [ch0, nchunk) of VW points read straight from global memory.
template <class Op, class T, class R, class Mdl, class K>
__device__ __forceinline__ void global_chunks(const KArgs& a, const K& k, int64_t ch0) {
  constexpr int VW = OpWidth<Op, T, R, Mdl>::VW;
  const int64_t nchunk = (a.n + VW - 1) / VW;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ch = ch0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunk; ch += stride) {
    const int64_t i0 = ch * VW;
    const int cnt = (a.n - i0 < VW) ? (int)(a.n - i0) : VW;
    const GlobalSrc<T, VW> src{a, i0, cnt};
    apply_chunk<Op, T, R, Mdl>(a, k, src, i0, cnt);
  }
}

template <class Op, class T, class R, class Mdl>
__global__ void __launch_bounds__(kThreads) k_pointwise(const __grid_constant__ KArgs a) {
  global_chunks<Op, T, R, Mdl>(a, Mdl::template make<R>(a), 0);
}

template <class Op, class T, class R, class Mdl>
__device__ __forceinline__ void staged_body(const KArgs& a) {
  constexpr int VW = OpWidth<Op, T, R, Mdl>::VW;
  constexpr int TILE = kThreads * VW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  T* buf = reinterpret_cast<T*>(smem_raw);  // [kStages][nin][TILE]
  const int nin = a.nin;
  const int tid = threadIdx.x;
  const int64_t ntiles = a.n / TILE;
  const uint32_t plane_bytes = TILE * sizeof(T);
  const auto k = Mdl::template make<R>(a);
  // polls per wait for a tile's copies (the drain after a timeout below keeps
  // the default limit, so every issued copy lands before the block exits)
  const int limit = a.wait_override > 0 ? a.wait_override - 1 : kWaitLimit;
  // The j-th tile of this block is tile blockIdx.x + j * gridDim.x, streamed
  // into stage j % kStages; its copy completes phase j / kStages of that
  // stage's mbarrier.
  int issued = 0;  // tiles whose copies thread 0 has issued
  auto issue = [&](int j) {
    const int s = j % kStages;
    const int64_t tile = blockIdx.x + (int64_t)j * gridDim.x;
    // (a tile out of range issues nothing; its wait then runs out)
    if (!FDBB_IDX_OK(a.dbg, tile >= 0 && (tile + 1) * TILE <= a.n && nin >= 1 && nin <= kMaxIn, tile * TILE)) return;
    mbar_expect_tx(&bars[s], nin * plane_bytes);
    for (int q = 0; q < nin; ++q)
      bulk_g2s(buf + ((size_t)s * nin + q) * TILE, inp<T>(a, q) + tile * TILE, plane_bytes, &bars[s]);
    ++issued;
  };
  auto has_tile = [&](int j) { return blockIdx.x + (int64_t)j * gridDim.x < ntiles; };
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < kStages && has_tile(j); ++j) issue(j);

  int j = 0;
  for (; has_tile(j); ++j) {
    const int s = j % kStages;
    const bool ok = mbar_wait(&bars[s], (uint32_t)(j / kStages) & 1u, limit);
    if (__syncthreads_or(!ok)) break;
#ifdef FDBB_DEBUG
    const SmemSrc<T, VW, TILE> src{buf + (size_t)s * nin * TILE + (size_t)tid * VW, nin, a.dbg};
#else
    const SmemSrc<T, VW, TILE> src{buf + (size_t)s * nin * TILE + (size_t)tid * VW};
#endif
    const int64_t i0 = (blockIdx.x + (int64_t)j * gridDim.x) * TILE + (int64_t)tid * VW;
    apply_chunk<Op, T, R, Mdl>(a, k, src, i0, VW);
    __syncthreads();  // the whole block is done with stage s: refill it
    if (tid == 0 && has_tile(j + kStages)) {
      fence_proxy_async();
      issue(j + kStages);
    }
  }
  if (has_tile(j)) {
    // A wait ran out: record it, wait (bounded again) for this block's copies
    // still in flight so that none lands after the block exits, and return.
    if (tid == 0) {
      atomicAdd(&g_wait_timeouts, 1u);
      for (int q = j; q < issued; ++q) mbar_wait(&bars[q % kStages], (uint32_t)(q / kStages) & 1u);
    }
    return;
  }
  // the ragged tail (fewer than TILE points) straight from global memory
  global_chunks<Op, T, R, Mdl>(a, k, ntiles * kThreads);
}

template <class Op, class T, class R, class Mdl>
__global__ void __launch_bounds__(kThreads) k_staged(const __grid_constant__ KArgs a) {
  staged_body<Op, T, R, Mdl>(a);
}

// The general-EOS double-word kernels, compiled for three resident blocks per
// SM (at most 85 registers per thread; left to itself the compiler takes 90
// and two blocks fit).
template <class Op, class T, class R, class Mdl>
__global__ void __launch_bounds__(kThreads, 3) k_staged3(const __grid_constant__ KArgs a) {
  staged_body<Op, T, R, Mdl>(a);
}
template <class R, class Mdl> constexpr bool kStaged3 = std::is_same<R, dw>::value && !std::is_same<Mdl, IdealModel>::value;

// The ideal-gas double-word fused pass, compiled for two resident blocks per
// SM (at most 128 registers per thread; left to itself the compiler may take
// more, and then one block fits).
template <class Op, class T, class R, class Mdl>
__global__ void __launch_bounds__(kThreads, 2) k_staged2(const __grid_constant__ KArgs a) {
  staged_body<Op, T, R, Mdl>(a);
}
template <class Op> struct IsFusedOp : std::false_type {};
template <int D, int d> struct IsFusedOp<OpFused<D, d>> : std::true_type {};
template <class Op, class R, class Mdl>
constexpr bool kStaged2 = IsFusedOp<Op>::value && std::is_same<R, dw>::value && std::is_same<Mdl, IdealModel>::value;

// Host: read and clear the timeout count of this translation unit.
inline unsigned int take_wait_timeouts_tu() {
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(zero));
  return v;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

// Persistent grid of the direct kernel: enough blocks to fill every SM at its
// occupancy, no more than there are chunks.
// Resident blocks per SM of `kern` with `smem` bytes of dynamic shared memory
// on the current device, cached per device in `cache` (one per kernel and
// shared-memory size).
template <class K>
int blocks_per_sm(K kern, size_t smem, std::atomic<int> (&cache)[kMaxDevices]) {
  const int slot = current_device_slot();
  if (slot >= 0) {
    const int v = cache[slot].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  if (b <= 0) b = 1;
  if (slot >= 0) cache[slot].store(b, std::memory_order_relaxed);
  return b;
}

template <class Op, class T, class R, class Mdl> cudaError_t launch_direct(const KArgs& a, cudaStream_t stream) {
  static std::atomic<int> bps_cache[kMaxDevices];
  const int bps = blocks_per_sm(k_pointwise<Op, T, R, Mdl>, 0, bps_cache);
  constexpr int VW = OpWidth<Op, T, R, Mdl>::VW;
  const int64_t nchunk = (a.n + VW - 1) / VW;
  const int64_t need = (nchunk + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)device_sm_count() * bps;
  const int grid = (int)(need < cap ? need : cap);
  k_pointwise<Op, T, R, Mdl><<<grid, kThreads, 0, stream>>>(a);
  record_launch(1, grid, kThreads, 0, VW);
  return cudaGetLastError();
}

// Staged kernel: kStages * nin planes of one tile in dynamic shared memory.
template <class Op, class T, class R, class Mdl> cudaError_t launch_staged(const KArgs& a, cudaStream_t stream) {
  constexpr int VW = OpWidth<Op, T, R, Mdl>::VW;
  constexpr int TILE = kThreads * VW;
  constexpr size_t kMaxSmem = (size_t)kStages * Op::kIn * TILE * sizeof(T);
  auto kern = [] {
    if constexpr (kStaged3<R, Mdl>)
      return k_staged3<Op, T, R, Mdl>;
    else if constexpr (kStaged2<Op, R, Mdl>)
      return k_staged2<Op, T, R, Mdl>;
    else
      return k_staged<Op, T, R, Mdl>;
  }();
  // the opt-in to more than 48 KB of dynamic shared memory is a property of
  // the kernel in each device's context: set it once per device
  static std::atomic<int> attr_set[kMaxDevices];
  const int slot = current_device_slot();
  if (slot < 0 || !attr_set[slot].load(std::memory_order_relaxed)) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    if (slot >= 0) attr_set[slot].store(1, std::memory_order_relaxed);
  }
  const size_t smem = (size_t)kStages * a.nin * TILE * sizeof(T);
  static std::atomic<int> bps_cache[Op::kIn + 1][kMaxDevices];  // blocks per SM for each nin
  const int bps = blocks_per_sm(kern, smem, bps_cache[a.nin]);
  const int64_t ntiles = a.n / TILE;
  const int64_t cap = (int64_t)device_sm_count() * bps;
  const int grid = (int)(ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap);
  kern<<<grid, kThreads, smem, stream>>>(a);
  record_launch(2, grid, kThreads, (int)smem, VW);
  return cudaGetLastError();
}

// The staged kernel pays off once every SM has a few tiles to stream, and
// while its two-stage ring leaves room for more than one block per SM; its
// bulk copies read device memory only (inputs in host memory take the direct
// kernel, kDirectOnly).
template <class Op, class T, class R, class Mdl = IdealModel>
cudaError_t launch_op(const KArgs& a, cudaStream_t stream) {
  constexpr int TILE = kThreads * OpWidth<Op, T, R, Mdl>::VW;
  const size_t ring = (size_t)kStages * a.nin * TILE * sizeof(T);
  if (!(a.flags & kDirectOnly) && a.n / TILE >= 4LL * device_sm_count() && a.nin >= 1 && a.nin <= Op::kIn &&
      ring <= (100u << 10))
    return launch_staged<Op, T, R, Mdl>(a, stream);
  return launch_direct<Op, T, R, Mdl>(a, stream);
}

// Dispatch on (op, dim, dir) for storage type T and compute type R.
template <int D, class T, class R> cudaError_t dispatch_dim(const LaunchReq& r, const KArgs& a) {
  const int d = r.dir;
  switch (r.op) {
    case OpKind::VMag2: return launch_op<OpVMag2<D>, T, R>(a, r.stream);
    case OpKind::Prim: return launch_op<OpPrim<D>, T, R>(a, r.stream);
    case OpKind::Cons: return launch_op<OpCons<D>, T, R>(a, r.stream);
    case OpKind::Eos: return launch_op<OpEos<D>, T, R>(a, r.stream);
    case OpKind::FluxAll: return launch_op<OpFlux<D, -1>, T, R>(a, r.stream);
    case OpKind::FluxPrimAll: return launch_op<OpFluxPrim<D, -1>, T, R>(a, r.stream);
    case OpKind::Temp: return launch_op<OpTemp<D>, T, R>(a, r.stream);
    default: break;
  }
#define FDBB_DIR_CASES(OPK, OPT, RT)                                                          \
  case OPK:                                                                                   \
    if (d == 0) return launch_op<OPT<D, 0>, T, RT>(a, r.stream);                              \
    if constexpr (D > 1)                                                                      \
      if (d == 1) return launch_op<OPT<D, (D > 1 ? 1 : 0)>, T, RT>(a, r.stream);              \
    if constexpr (D > 2)                                                                      \
      if (d == 2) return launch_op<OPT<D, (D > 2 ? 2 : 0)>, T, RT>(a, r.stream);              \
    return cudaErrorInvalidValue;
  switch (r.op) {
    FDBB_DIR_CASES(OpKind::Riemann, OpRiemann, R)
    FDBB_DIR_CASES(OpKind::Flux, OpFlux, R)
    FDBB_DIR_CASES(OpKind::Jac, OpJac, R)
    FDBB_DIR_CASES(OpKind::Fused, OpFused, R)
    FDBB_DIR_CASES(OpKind::Vjp, OpVjp, R)
    FDBB_DIR_CASES(OpKind::RoeFlux, OpRoeFlux, R)
    FDBB_DIR_CASES(OpKind::FluxPrim, OpFluxPrim, R)
    FDBB_DIR_CASES(OpKind::JacPrim, OpJacPrim, R)
    case OpKind::RoeCharFwd:
      if (d == 0) return launch_op<OpRoeChar<D, 0, false>, T, R>(a, r.stream);
      if constexpr (D > 1)
        if (d == 1) return launch_op<OpRoeChar<D, (D > 1 ? 1 : 0), false>, T, R>(a, r.stream);
      if constexpr (D > 2)
        if (d == 2) return launch_op<OpRoeChar<D, (D > 2 ? 2 : 0), false>, T, R>(a, r.stream);
      return cudaErrorInvalidValue;
    case OpKind::RoeCharInv:
      if (d == 0) return launch_op<OpRoeChar<D, 0, true>, T, R>(a, r.stream);
      if constexpr (D > 1)
        if (d == 1) return launch_op<OpRoeChar<D, (D > 1 ? 1 : 0), true>, T, R>(a, r.stream);
      if constexpr (D > 2)
        if (d == 2) return launch_op<OpRoeChar<D, (D > 2 ? 2 : 0), true>, T, R>(a, r.stream);
      return cudaErrorInvalidValue;
    case OpKind::CharFwd:
      if (d == 0) return launch_op<OpChar<D, 0, false>, T, R>(a, r.stream);
      if constexpr (D > 1)
        if (d == 1) return launch_op<OpChar<D, (D > 1 ? 1 : 0), false>, T, R>(a, r.stream);
      if constexpr (D > 2)
        if (d == 2) return launch_op<OpChar<D, (D > 2 ? 2 : 0), false>, T, R>(a, r.stream);
      return cudaErrorInvalidValue;
    case OpKind::CharInv:
      if (d == 0) return launch_op<OpChar<D, 0, true>, T, R>(a, r.stream);
      if constexpr (D > 1)
        if (d == 1) return launch_op<OpChar<D, (D > 1 ? 1 : 0), true>, T, R>(a, r.stream);
      if constexpr (D > 2)
        if (d == 2) return launch_op<OpChar<D, (D > 2 ? 2 : 0), true>, T, R>(a, r.stream);
      return cudaErrorInvalidValue;
    default: break;
  }
#undef FDBB_DIR_CASES
  return cudaErrorInvalidValue;
}

template <class T, class R> cudaError_t dispatch(const LaunchReq& r, const KArgs& a) {
  switch (r.dim) {
    case 1: return dispatch_dim<1, T, R>(r, a);
    case 2: return dispatch_dim<2, T, R>(r, a);
    case 3: return dispatch_dim<3, T, R>(r, a);
    default: return cudaErrorInvalidValue;
  }
}

// General-EOS blocks for EOS model Mdl, storage T computed in R (T's own IEEE
// type, or double-word for double): every block whose formulas the EOS enters, except the Riemann
// invariants and the Roe-averaged forms, which have no closed form for a
// general EOS.
template <int D, class T, class R, class Mdl> cudaError_t dispatch_eos_dim(const LaunchReq& r, const KArgs& a) {
  const int d = r.dir;
  switch (r.op) {
    case OpKind::Prim: return launch_op<OpPrim<D>, T, R, Mdl>(a, r.stream);
    case OpKind::Cons: return launch_op<OpCons<D>, T, R, Mdl>(a, r.stream);
    case OpKind::Eos: return launch_op<OpEos<D>, T, R, Mdl>(a, r.stream);
    case OpKind::FluxAll: return launch_op<OpFlux<D, -1>, T, R, Mdl>(a, r.stream);
    case OpKind::FluxPrimAll: return launch_op<OpFluxPrim<D, -1>, T, R, Mdl>(a, r.stream);
    case OpKind::Temp: return launch_op<OpTemp<D>, T, R, Mdl>(a, r.stream);
    default: break;
  }
#define FDBB_EOS_DIR_CASES(OPK, ...)                                                              \
  case OPK:                                                                                       \
    if (d == 0) return launch_op<__VA_ARGS__<D, 0>, T, R, Mdl>(a, r.stream);                      \
    if constexpr (D > 1)                                                                          \
      if (d == 1) return launch_op<__VA_ARGS__<D, (D > 1 ? 1 : 0)>, T, R, Mdl>(a, r.stream);      \
    if constexpr (D > 2)                                                                          \
      if (d == 2) return launch_op<__VA_ARGS__<D, (D > 2 ? 2 : 0)>, T, R, Mdl>(a, r.stream);      \
    return cudaErrorInvalidValue;
  switch (r.op) {
    FDBB_EOS_DIR_CASES(OpKind::Flux, OpFlux)
    FDBB_EOS_DIR_CASES(OpKind::Jac, OpJac)
    FDBB_EOS_DIR_CASES(OpKind::Fused, OpFused)
    FDBB_EOS_DIR_CASES(OpKind::Vjp, OpVjp)
    FDBB_EOS_DIR_CASES(OpKind::FluxPrim, OpFluxPrim)
    FDBB_EOS_DIR_CASES(OpKind::JacPrim, OpJacPrim)
    FDBB_EOS_DIR_CASES(OpKind::CharFwd, OpCharFwd)
    FDBB_EOS_DIR_CASES(OpKind::CharInv, OpCharInv)
    default: break;
  }
#undef FDBB_EOS_DIR_CASES
  return cudaErrorInvalidValue;
}

template <class T, class R, class Mdl> cudaError_t dispatch_eos_model(const LaunchReq& r, const KArgs& a) {
  switch (r.dim) {
    case 1: return dispatch_eos_dim<1, T, R, Mdl>(r, a);
    case 2: return dispatch_eos_dim<2, T, R, Mdl>(r, a);
    case 3: return dispatch_eos_dim<3, T, R, Mdl>(r, a);
    default: return cudaErrorInvalidValue;
  }
}

template <class T, class R> cudaError_t dispatch_eos(const LaunchReq& r, const KArgs& a) {
  switch (r.eos) {
    case EosKind::Nasg: return dispatch_eos_model<T, R, NasgModel>(r, a);
    case EosKind::Vdw: return dispatch_eos_model<T, R, VdwModel>(r, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdbb
