// fdbb_kernels.cuh -- one fused grid-stride kernel per building block.
//
// Every kernel is k_pointwise<Op, T, R>: a persistent grid (a multiple of the
// SM count) strides over chunks of VW points; Op::apply loads the chunk's input
// planes (storage type T), converts them to the compute type R, evaluates its
// expressions in registers and stores its output planes.  No temporaries touch
// memory.
//
// apply() returns false -- before storing anything -- when the double-word
// range guard fails; the kernel then recomputes that chunk in native FP64.
#pragma once

#include <type_traits>

#include "fdbb_device.cuh"
#include "fdbb_internal.h"

namespace fdbb {

constexpr int kThreads = 256;

template <class T> __device__ __forceinline__ const T* inp(const KArgs& a, int k) {
  return static_cast<const T*>(a.in[k]);
}
template <class T> __device__ __forceinline__ T* outp(const KArgs& a, int k) {
  return static_cast<T*>(a.out[k]);
}

template <class R> __device__ __forceinline__ Consts<R> consts(const KArgs& a);
template <> __device__ __forceinline__ Consts<double> consts<double>(const KArgs& a) {
  return {a.kd[0], a.kd[1], a.kd[2], a.kd[3], a.kd[4], a.kd[5]};
}
template <> __device__ __forceinline__ Consts<float> consts<float>(const KArgs& a) {
  return {a.kf[0], a.kf[1], a.kf[2], a.kf[3], a.kf[4], a.kf[5]};
}
template <> __device__ __forceinline__ Consts<dw> consts<dw>(const KArgs& a) {
  return {dw(a.kf[0], a.kl[0]), dw(a.kf[1], a.kl[1]), dw(a.kf[2], a.kl[2]),
          dw(a.kf[3], a.kl[3]), dw(a.kf[4], a.kl[4]), dw(a.kf[5], a.kl[5])};
}

// Conservative state of VW points from input planes base..base+D+1.
template <class T, int VW, int D, class R, class G>
__device__ __forceinline__ void load_U(const KArgs& a, int base, int64_t i0, int cnt, Pt<R, D> (&s)[VW], G& g) {
  typename Storage<T>::L raw[VW];
  load_raw<T, VW>(inp<T>(a, base), i0, cnt, raw, 1.0f);
#pragma unroll
  for (int j = 0; j < VW; ++j) {
    s[j].rho = to_compute<R, G>(raw[j], g);
    if constexpr (std::is_same<R, dw>::value) s[j].raw.rho = raw[j];
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    load_raw<T, VW>(inp<T>(a, base + 1 + i), i0, cnt, raw, 0.0f);
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      s[j].m[i] = to_compute<R, G>(raw[j], g);
      if constexpr (std::is_same<R, dw>::value) s[j].raw.m[i] = raw[j];
    }
  }
  load_raw<T, VW>(inp<T>(a, base + D + 1), i0, cnt, raw, 1.0f);
#pragma unroll
  for (int j = 0; j < VW; ++j) s[j].rE = to_compute<R, G>(raw[j], g);
}

// nv planes of a second input field (W or G) from planes base..base+nv-1,
// as w[point][component].
template <class T, int VW, int NV, class R, class G>
__device__ __forceinline__ void load_field(const KArgs& a, int base, int64_t i0, int cnt, R (&w)[VW][NV], G& g) {
  R x[VW];
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    load<T, VW, R>(inp<T>(a, base + c), i0, cnt, x, 0.0f, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) w[j][c] = x[j];
  }
}

// Store y[point][component] into output planes base..base+NV-1.
template <class T, int VW, int NV, class R>
__device__ __forceinline__ void store_field(const KArgs& a, int base, int64_t i0, int cnt, const R (&y)[VW][NV]) {
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    T* o = outp<T>(a, base + c);
    if (!o) continue;
    R x[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) x[j] = y[j][c];
    store<T, VW, R>(o, i0, cnt, x);
  }
}

template <int VW, int D, class R, class G>
__device__ __forceinline__ void derive_all(Pt<R, D> (&s)[VW], const Consts<R>& k, G& g) {
#pragma unroll
  for (int j = 0; j < VW; ++j) derive(s[j], k, g);
}

// Flux column d into output planes base..base+nv-1.  Component 0 is the input
// momentum m_d itself, stored bit for bit.
template <class T, int VW, int D, int d, class R>
__device__ __forceinline__ void emit_flux(const KArgs& a, int base, int64_t i0, int cnt, const Pt<R, D> (&s)[VW]) {
#pragma unroll
  for (int c = 0; c < D + 2; ++c) {
    T* o = outp<T>(a, base + c);
    if (!o) continue;
    if constexpr (std::is_same<R, dw>::value) {
      if (c == 0) {  // F_d[0] = m_d: the input itself, bit for bit
        double raw[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) raw[j] = s[j].raw.m[d];
        store_raw<T, VW>(o, i0, cnt, raw);
        continue;
      }
    }
    R x[VW];
#pragma unroll
    for (int j = 0; j < VW; ++j) x[j] = flux_comp<D, d>(s[j], c);
    store<T, VW, R>(o, i0, cnt, x);
  }
}

// Jacobian A_d into output planes base..base+nv*nv-1 (row-major).
template <class T, int VW, int D, int d, class R>
__device__ __forceinline__ void emit_jac(const KArgs& a, int base, int64_t i0, int cnt, const Pt<R, D> (&s)[VW],
                                         const Consts<R>& k) {
  constexpr int nv = D + 2;
#pragma unroll
  for (int row = 0; row < nv; ++row) {
#pragma unroll
    for (int col = 0; col < nv; ++col) {
      T* o = outp<T>(a, base + row * nv + col);
      if (!o) continue;
      R x[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) x[j] = jac_entry<D, d>(s[j], k, row, col);
      store<T, VW, R>(o, i0, cnt, x);
    }
  }
}

// ---------------------------------------------------------------------------
// Ops
// ---------------------------------------------------------------------------

// |v|^2 = (sum m_i^2) / (rho rho)  (paper section 3, Eq. (2)).
template <int D> struct OpVMag2 {
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>&, int64_t i0, int cnt) {
    typename GuardOf<R>::type g;
    R rho[VW], m[VW], num[VW];
    load<T, VW, R>(inp<T>(a, 0), i0, cnt, rho, 1.0f, g);
    load<T, VW, R>(inp<T>(a, 1), i0, cnt, m, 0.0f, g);
#pragma unroll
    for (int j = 0; j < VW; ++j) num[j] = m[j] * m[j];
#pragma unroll
    for (int i = 1; i < D; ++i) {
      load<T, VW, R>(inp<T>(a, 1 + i), i0, cnt, m, 0.0f, g);
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
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    derive_all<VW, D>(s, k, g);
    if (!g.ok) return false;
    R x[VW];
    if constexpr (std::is_same<R, dw>::value) {
      double raw[VW];
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

// U = (rho, rho v, p/(gamma-1) + rho |v|^2 / 2) from V.
template <int D> struct OpCons {
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    typename GuardOf<R>::type g;
    R rho[VW], v[D][VW], p[VW], x[VW];
    typename Storage<T>::L rho_raw[VW];
    load_raw<T, VW>(inp<T>(a, 0), i0, cnt, rho_raw, 1.0f);
#pragma unroll
    for (int j = 0; j < VW; ++j) rho[j] = to_compute<R>(rho_raw[j], g);
#pragma unroll
    for (int i = 0; i < D; ++i) load<T, VW, R>(inp<T>(a, 1 + i), i0, cnt, v[i], 0.0f, g);
    load<T, VW, R>(inp<T>(a, D + 1), i0, cnt, p, 1.0f, g);
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
    for (int j = 0; j < VW; ++j) x[j] = fma_(p[j], k.ia1, R(0.5f) * rho[j] * v2[j]);
    store<T, VW, R>(outp<T>(a, D + 1), i0, cnt, x);
    return true;
  }
};

// p and c.
template <int D> struct OpEos {
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    derive_all<VW, D>(s, k, g);
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
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    derive_all<VW, D>(s, k, g);
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
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    derive_all<VW, D>(s, k, g);
    if (!g.ok) return false;
    if constexpr (d >= 0) {
      emit_flux<T, VW, D, d>(a, 0, i0, cnt, s);
    } else {
      emit_flux<T, VW, D, 0>(a, 0, i0, cnt, s);
      if constexpr (D > 1) emit_flux<T, VW, D, 1>(a, D + 2, i0, cnt, s);
      if constexpr (D > 2) emit_flux<T, VW, D, 2>(a, 2 * (D + 2), i0, cnt, s);
    }
    return true;
  }
};

template <int D, int d> struct OpJac {
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    derive_all<VW, D>(s, k, g);
    if (!g.ok) return false;
    emit_jac<T, VW, D, d>(a, 0, i0, cnt, s, k);
    return true;
  }
};

template <int D, int d, bool INV> struct OpChar {
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    R w[VW][nv], y[VW][nv];
    load_field<T, VW, nv>(a, nv, i0, cnt, w, g);
    derive_all<VW, D>(s, k, g);
    if (!g.ok) return false;
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      if constexpr (INV)
        char_inv<D, d>(s[j], k, w[j], y[j]);
      else
        char_fwd<D, d>(s[j], k, w[j], y[j]);
    }
    store_field<T, VW, nv>(a, 0, i0, cnt, y);
    return true;
  }
};

// All flux columns (planes 0..D*nv-1), A_dj (D*nv .. D*nv+nv^2-1) and
// L_dj W (last nv planes) in one pass; inputs U (planes 0..nv-1), W (nv..2nv-1).
template <int D, int dj> struct OpFused {
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    R w[VW][nv];
    const bool want_y = a.in[nv] != nullptr;
    if (want_y) load_field<T, VW, nv>(a, nv, i0, cnt, w, g);
    derive_all<VW, D>(s, k, g);
    if (!g.ok) return false;
    emit_flux<T, VW, D, 0>(a, 0, i0, cnt, s);
    if constexpr (D > 1) emit_flux<T, VW, D, 1>(a, nv, i0, cnt, s);
    if constexpr (D > 2) emit_flux<T, VW, D, 2>(a, 2 * nv, i0, cnt, s);
    emit_jac<T, VW, D, dj>(a, D * nv, i0, cnt, s, k);
    if (want_y) {
      R y[VW][nv];
#pragma unroll
      for (int j = 0; j < VW; ++j) char_fwd<D, dj>(s[j], k, w[j], y[j]);
      store_field<T, VW, nv>(a, D * nv + nv * nv, i0, cnt, y);
    }
    return true;
  }
};

template <int D, int d> struct OpVjp {
  template <class T, int VW, class R>
  static __device__ __forceinline__ bool apply(const KArgs& a, const Consts<R>& k, int64_t i0, int cnt) {
    constexpr int nv = D + 2;
    typename GuardOf<R>::type g;
    Pt<R, D> s[VW];
    load_U<T, VW, D>(a, 0, i0, cnt, s, g);
    R gg[VW][nv], y[VW][nv];
    load_field<T, VW, nv>(a, nv, i0, cnt, gg, g);
    derive_all<VW, D>(s, k, g);
    if (!g.ok) return false;
#pragma unroll
    for (int j = 0; j < VW; ++j) flux_vjp_pt<D, d>(s[j], k, gg[j], y[j]);
    store_field<T, VW, nv>(a, 0, i0, cnt, y);
    return true;
  }
};

// ---------------------------------------------------------------------------
// The kernel and its launcher
// ---------------------------------------------------------------------------
template <class Op, class T, class R>
__global__ void __launch_bounds__(kThreads) k_pointwise(const __grid_constant__ KArgs a) {
  constexpr int VW = Width<T, R>::VW;
  const Consts<R> k = consts<R>(a);
  const int64_t nchunk = (a.n + VW - 1) / VW;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunk; ch += stride) {
    const int64_t i0 = ch * VW;
    const int cnt = (a.n - i0 < VW) ? (int)(a.n - i0) : VW;
    if constexpr (std::is_same<R, dw>::value) {
      // double-word fast path; chunks outside its range run in native FP64
      if (!Op::template apply<T, VW, dw>(a, k, i0, cnt))
        Op::template apply<T, VW, double>(a, consts<double>(a), i0, cnt);
    } else {
      Op::template apply<T, VW, R>(a, k, i0, cnt);
    }
  }
}

// Persistent grid: enough blocks to fill every SM at the kernel's occupancy,
// but no more blocks than there are chunks to process.
template <class Op, class T, class R> cudaError_t launch_op(const KArgs& a, cudaStream_t stream) {
  static const int blocks_per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pointwise<Op, T, R>, kThreads, 0) != cudaSuccess) b = 1;
    return b > 0 ? b : 1;
  }();
  constexpr int VW = Width<T, R>::VW;
  const int64_t nchunk = (a.n + VW - 1) / VW;
  const int64_t need = (nchunk + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)device_sm_count() * blocks_per_sm;
  const int grid = (int)(need < cap ? need : cap);
  k_pointwise<Op, T, R><<<grid, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
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
    default: break;
  }
  // The inverse characteristic transform adds input components directly
  // (a1 + a2 + an); in double-word arithmetic such sums of exact inputs are
  // not accurate relative to their own magnitude, so it always runs in the
  // storage's own IEEE type.
  using RI = typename std::conditional<std::is_same<R, dw>::value, double, R>::type;
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
    case OpKind::CharFwd:
      if (d == 0) return launch_op<OpChar<D, 0, false>, T, R>(a, r.stream);
      if constexpr (D > 1)
        if (d == 1) return launch_op<OpChar<D, (D > 1 ? 1 : 0), false>, T, R>(a, r.stream);
      if constexpr (D > 2)
        if (d == 2) return launch_op<OpChar<D, (D > 2 ? 2 : 0), false>, T, R>(a, r.stream);
      return cudaErrorInvalidValue;
    case OpKind::CharInv:
      if (d == 0) return launch_op<OpChar<D, 0, true>, T, RI>(a, r.stream);
      if constexpr (D > 1)
        if (d == 1) return launch_op<OpChar<D, (D > 1 ? 1 : 0), true>, T, RI>(a, r.stream);
      if constexpr (D > 2)
        if (d == 2) return launch_op<OpChar<D, (D > 2 ? 2 : 0), true>, T, RI>(a, r.stream);
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

}  // namespace fdbb
