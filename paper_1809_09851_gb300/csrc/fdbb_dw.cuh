// fdbb_dw.cuh -- double-word ("float-float") arithmetic for FP64-storage
// kernels on GB300.
//
// GB300 executes FP64 FMA, FP64<->FP32 conversion and every other FP64-pipe
// instruction at 1/64 of the FP32 rate (about 2 per clock per SM).  The fused
// 3D pass needs ~70 FP64 operations per point, which makes it FP64-bound at
// about half of the HBM roofline.  A double-word number x = hi + lo (two
// floats, |lo| <= ulp(hi)) carries a ~47-bit significand; its arithmetic runs
// on the FP32 pipe and the conversions from and to IEEE double are done with
// integer bit operations, so no FP64-pipe instruction is needed on the fast
// path.
//
// Algorithms (all error-free-transform based):
//   TwoSum (Knuth), Fast2Sum (Dekker), TwoProd via FMA;
//   addition  = "SloppyDWPlusDW", multiplication = "DWTimesDW1" of
//   M. Joldes, J.-M. Muller, V. Popescu, "Tight and rigorous error bounds for
//   basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017;
//   reciprocal / reciprocal square root = one Newton step from the hardware
//   approximation with the residual formed exactly by FMA.
// The sloppy addition is accurate to ~4u^2 (|a| + |b|) (u = 2^-24) rather than
// relative to |a + b|; with respect to the running-error scale of the
// formulas (which contains |a| + |b| whenever an operand is itself computed)
// this is the same order as the other operations.  Sums of two *exact inputs*
// are never formed in double-word arithmetic (the inverse characteristic
// transform, the only block that adds inputs directly, stays in FP64).
//
// Range: the fast path is taken only where every input and derived
// quantity is 0 or has magnitude in [2^-24, 2^24] (DwGuard); products of
// up to four such factors then stay far inside the normal float range, so no
// low word underflows.  A point outside it is recomputed in native FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdbb {

struct dw {
  float hi, lo;
  dw() = default;
  __device__ __forceinline__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ constexpr dw(float h) : hi(h), lo(0.0f) {}
  __device__ __forceinline__ constexpr dw(double) = delete;
  __device__ __forceinline__ constexpr dw(int h) : hi(static_cast<float>(h)), lo(0.0f) {}
};

// s + e == a + b exactly (Knuth).
__device__ __forceinline__ void dw_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ void dw_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dw operator-(dw a) { return dw(-a.hi, -a.lo); }

__device__ __forceinline__ dw operator+(dw a, dw b) {
  float s, e;
  dw_two_sum(a.hi, b.hi, s, e);
  const float v = __fadd_rn(a.lo, b.lo);
  const float w = __fadd_rn(e, v);
  dw z;
  dw_fast_two_sum(s, w, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ dw operator-(dw a, dw b) { return a + (-b); }

__device__ __forceinline__ dw operator*(dw a, dw b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  const float t = __fmul_rn(a.hi, b.lo);
  const float c = __fmaf_rn(a.lo, b.hi, t);
  const float l = __fadd_rn(pe, c);
  dw z;
  dw_fast_two_sum(p, l, z.hi, z.lo);
  return z;
}

// a * b + c with one renormalisation.
__device__ __forceinline__ dw fma_(dw a, dw b, dw c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  float s, se;
  dw_two_sum(p, c.hi, s, se);
  float t = __fmaf_rn(a.hi, b.lo, pe);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fadd_rn(t, c.lo);
  t = __fadd_rn(t, se);
  dw z;
  dw_fast_two_sum(s, t, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ float dw_rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float dw_rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 1/y: r0 ~ 1/y.hi, e = 1 - y r0 (exact residual of the high word by FMA),
// 1/y = r0 (1 + e + e^2 + ...).
__device__ __forceinline__ dw rcp_(dw y) {
  const float r0 = dw_rcp_approx(y.hi);
  float e = __fmaf_rn(-y.hi, r0, 1.0f);
  e = __fmaf_rn(-y.lo, r0, e);
  const float c = __fmaf_rn(e, e, e);
  dw z;
  dw_fast_two_sum(r0, __fmul_rn(r0, c), z.hi, z.lo);
  return z;
}

// 1/sqrt(x): y0 ~ 1/sqrt(x.hi), m = x y0^2 - 1 (formed with TwoProd and FMA),
// 1/sqrt(x) = y0 (1 - m/2 + 3 m^2 / 8 - ...).
__device__ __forceinline__ dw rsqrt_(dw x) {
  const float y0 = dw_rsqrt_approx(x.hi);
  const float q = __fmul_rn(y0, y0);
  const float qe = __fmaf_rn(y0, y0, -q);
  float m = __fmaf_rn(x.hi, q, -1.0f);
  m = __fmaf_rn(x.hi, qe, m);
  m = __fmaf_rn(x.lo, q, m);
  const float c = __fmaf_rn(0.375f, m, -0.5f);
  dw z;
  dw_fast_two_sum(y0, __fmul_rn(y0, __fmul_rn(m, c)), z.hi, z.lo);
  return z;
}

__device__ __forceinline__ dw operator/(dw a, dw b) { return a * rcp_(b); }

__device__ __forceinline__ dw abs_(dw x) { return x.hi < 0.0f ? -x : x; }

__device__ __forceinline__ dw sqrt_(dw x) {
  if (x.hi == 0.0f) return dw(0.0f);
  return x * rsqrt_(x);
}

// ---------------------------------------------------------------------------
// Conversions between IEEE double and double-word, in integer arithmetic.
// ---------------------------------------------------------------------------

// Range guard of the double-word fast path: every checked value is 0 or has
// magnitude in [2^-24, 2^24].
struct DwGuard {
  bool ok = true;
  __device__ __forceinline__ void check(dw x) {
    const float a = fabsf(x.hi);
    ok &= ((a >= 0x1p-24f) & (a <= 0x1p24f)) | (a == 0.0f);  // NaN compares false
  }
};

// Two instruction sequences for each conversion, with the same results up to
// the sign of a zero and values below 2^-82 (where both stay within |lo| of
// hi + lo).  They differ in how a zero is handled -- by clamping the exponent
// arithmetic (kClamp, fewer instructions) or by selects at the end (kSelect)
// -- and so in how the compiler schedules them: which is faster depends on
// the register pressure of the kernel (the table at DwConvOf in
// fdbb_kernels.cuh).
enum class DwConv { kClamp, kSelect };

// Split a double into hi (its leading 24 significant bits, truncated) and lo
// (the next 23 bits, exact in float): |x - (hi + lo)| <= 2^-47 |x|.  The
// guard records whether x is 0 or 2^-24 <= |x| < 2^24 (tested on the double's
// own exponent field, since outside 2^-102 <= |x| < 2^128 the split itself is
// meaningless).
template <DwConv C = DwConv::kClamp>
__device__ __forceinline__ dw dw_from_double(double x, DwGuard& g) {
  const uint32_t H = static_cast<uint32_t>(__double2hiint(x));
  const uint32_t L = static_cast<uint32_t>(__double2loint(x));
  if constexpr (C == DwConv::kClamp) {
    const uint32_t mag = H & 0x7FFFFFFFu;
    const bool zero = (mag | L) == 0u;
    g.ok &= zero | ((mag - (999u << 20)) < (48u << 20));       // 0 or 2^-24 <= |x| < 2^24
    // exponent 1023 -> 127 bias, clamped at 0: a zero gives hi = +-0 and
    // lo = 0 (other values below 2^-127 fail the guard)
    const int32_t tb = static_cast<int32_t>(mag) - static_cast<int32_t>(896u << 20);
    const uint32_t t = static_cast<uint32_t>(tb > 0 ? tb : 0);
    const uint32_t hb = __funnelshift_l(L, t, 3) | (H & 0x80000000u);  // sign | exp | top 23 mantissa bits
    const uint32_t base = (hb & 0xFF800000u) - (23u << 23);     // sign | 2^(e-23)
    const uint32_t yb = base | ((L >> 6) & 0x007FFFFFu);        // 2^(e-23) * (1 + next 23 bits)
    return dw(__uint_as_float(hb), __fsub_rn(__uint_as_float(yb), __uint_as_float(base)));
  } else {
    const bool zero = ((H << 1) | L) == 0u;
    const uint32_t E = (H >> 20) & 0x7FFu;
    g.ok &= zero | ((E - 999u) < 48u);
    const uint32_t sign = H & 0x80000000u;
    const uint32_t t = (H & 0x7FFFFFFFu) - (896u << 20);
    const uint32_t hb = __funnelshift_l(L, t, 3) | sign;
    const uint32_t base = (hb & 0xFF800000u) - (23u << 23);
    const uint32_t yb = base | ((L >> 6) & 0x007FFFFFu);
    const float lo = __fsub_rn(__uint_as_float(yb), __uint_as_float(base));
    return dw(zero ? 0.0f : __uint_as_float(hb), zero ? 0.0f : lo);
  }
}

__device__ __forceinline__ dw dw_from_double_unchecked(double x) {
  DwGuard g;
  return dw_from_double(x, g);
}

// hi + lo rounded to a double: the double of hi is built from its bit pattern
// and lo is added as an integer number of units of 2^(e_hi - 45) (|lo| <
// 2^(e_hi - 23), so the count fits the float magic-number rounding range).
// Error <= 2^-46 |x| for |x| >= 2^-82; below, where the scale 2^(45 - e_hi)
// is not a normal float, at most |lo|.  When hi is a power of two and the
// correction is negative the result lies in the binade below, whose ulp is
// half as large.
template <DwConv C = DwConv::kClamp>
__device__ __forceinline__ double dw_to_double(dw x) {
  const uint32_t f = __float_as_uint(x.hi);
  if constexpr (C == DwConv::kClamp) {
    const uint32_t ebits = f & 0x7F800000u;
    // sign, the 8 exponent bits rebiased by 896 (not for a zero or subnormal
    // hi, whose double is then 0 or below 2^-1022) and the 23 mantissa bits
    const uint32_t H = (static_cast<uint32_t>(static_cast<int32_t>(f) >> 3) & 0x8FFFFFFFu) +
                       (ebits != 0u ? (896u << 20) : 0u);
    const uint32_t L = f << 29;
    // the scale is capped at 2^127: for |hi| < 2^-82 less than lo is added,
    // and a zero hi (with its zero lo) adds nothing
    const uint32_t sb = min((299u << 23) - ebits, 0x7F000000u);
    const float k = __fmaf_rn(x.lo, __uint_as_float(sb | (f & 0x80000000u)), 12582912.0f);  // 1.5 * 2^23
    const int32_t ki = static_cast<int32_t>(__float_as_uint(k)) - 0x4B400000;
    const int32_t unit = ((f & 0x007FFFFFu) == 0u && ki < 0) ? 256 : 128;
    const int64_t bits = static_cast<int64_t>((static_cast<uint64_t>(H) << 32) | L);
    return __longlong_as_double(bits + static_cast<int64_t>(ki) * unit);
  } else {
    const uint32_t mag = f & 0x7FFFFFFFu;
    const uint32_t sign = f & 0x80000000u;
    const uint32_t H = ((mag >> 3) + (896u << 20)) | sign;
    const uint32_t L = f << 29;
    const int64_t bits = static_cast<int64_t>((static_cast<uint64_t>(H) << 32) | L);
    const uint32_t ebits = mag & 0x7F800000u;
    // below |hi| = 2^-82 lo is dropped
    const float scale = __uint_as_float(((299u << 23) - ebits) | sign);
    const float k = __fmaf_rn(x.lo, scale, 12582912.0f);
    const int32_t ki0 = static_cast<int32_t>(__float_as_uint(k)) - 0x4B400000;
    const int32_t ki = ebits >= (45u << 23) ? ki0 : 0;
    const int64_t unit = ((mag & 0x007FFFFFu) == 0u && ki < 0) ? 256 : 128;
    const int64_t out = bits + static_cast<int64_t>(ki) * unit;
    // |hi| < 2^-126 (zero or subnormal): a signed zero
    return mag < 0x00800000u ? __hiloint2double(static_cast<int>(sign), 0) : __longlong_as_double(out);
  }
}


// x^y through FP64 (used only for the optional entropy output).
__device__ __forceinline__ dw pow_(dw x, dw y) {
  return dw_from_double_unchecked(pow(dw_to_double(x), dw_to_double(y)));
}

// ---------------------------------------------------------------------------
// Two double-word values in packed FP32x2 registers (sm_100 and later).
// Lane x and lane y are two independent points; every operation is the
// double-word operation above, lane by lane, with each FP32 step issued as one
// packed instruction (FADD2 / FMUL2 / FFMA2) for both points.  Each lane
// rounds exactly as the scalar operation, so a lane's result equals the
// double-word result bit for bit.
// ---------------------------------------------------------------------------
struct dw2 {
  float2 hi, lo;
  dw2() = default;
  __device__ __forceinline__ dw2(float2 h, float2 l) : hi(h), lo(l) {}
  __device__ __forceinline__ dw2(float h) : hi(make_float2(h, h)), lo(make_float2(0.0f, 0.0f)) {}
  __device__ __forceinline__ dw2(int h) : dw2(static_cast<float>(h)) {}
  __device__ __forceinline__ dw2(double) = delete;
};

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as (-1) b + a: the product is exact, so one rounding as in a subtraction
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void dw2_fast_two_sum(float2 a, float2 b, float2& s, float2& e) {
  s = p_add(a, b);
  e = p_sub(b, p_sub(s, a));
}

__device__ __forceinline__ dw2 operator-(dw2 a) { return dw2(p_neg(a.hi), p_neg(a.lo)); }

__device__ __forceinline__ dw2 operator+(dw2 a, dw2 b) {
  const float2 s = p_add(a.hi, b.hi);
  const float2 bb = p_sub(s, a.hi);
  const float2 e = p_add(p_sub(a.hi, p_sub(s, bb)), p_sub(b.hi, bb));
  const float2 w = p_add(e, p_add(a.lo, b.lo));
  dw2 z;
  dw2_fast_two_sum(s, w, z.hi, z.lo);
  return z;
}

// a + (-b) of the scalar type with the negations folded in:
// (-b) - bb = -(b + bb) and a.lo + (-b.lo) = a.lo - b.lo exactly.
__device__ __forceinline__ dw2 operator-(dw2 a, dw2 b) {
  const float2 s = p_sub(a.hi, b.hi);
  const float2 bb = p_sub(s, a.hi);
  const float2 e = p_sub(p_sub(a.hi, p_sub(s, bb)), p_add(b.hi, bb));
  const float2 w = p_add(e, p_sub(a.lo, b.lo));
  dw2 z;
  dw2_fast_two_sum(s, w, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ dw2 operator*(dw2 a, dw2 b) {
  const float2 p = p_mul(a.hi, b.hi);
  const float2 pe = p_fma(a.hi, b.hi, p_neg(p));
  const float2 t = p_mul(a.hi, b.lo);
  const float2 c = p_fma(a.lo, b.hi, t);
  const float2 l = p_add(pe, c);
  dw2 z;
  dw2_fast_two_sum(p, l, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ dw2 fma_(dw2 a, dw2 b, dw2 c) {
  const float2 p = p_mul(a.hi, b.hi);
  const float2 pe = p_fma(a.hi, b.hi, p_neg(p));
  const float2 s = p_add(p, c.hi);
  const float2 bb = p_sub(s, p);
  const float2 se = p_add(p_sub(p, p_sub(s, bb)), p_sub(c.hi, bb));
  float2 t = p_fma(a.hi, b.lo, pe);
  t = p_fma(a.lo, b.hi, t);
  t = p_add(t, c.lo);
  t = p_add(t, se);
  dw2 z;
  dw2_fast_two_sum(s, t, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ dw2 rcp_(dw2 y) {
  const float2 r0 = make_float2(dw_rcp_approx(y.hi.x), dw_rcp_approx(y.hi.y));
  float2 e = p_fma(p_neg(y.hi), r0, make_float2(1.0f, 1.0f));
  e = p_fma(p_neg(y.lo), r0, e);
  const float2 c = p_fma(e, e, e);
  dw2 z;
  dw2_fast_two_sum(r0, p_mul(r0, c), z.hi, z.lo);
  return z;
}

__device__ __forceinline__ dw2 operator/(dw2 a, dw2 b) { return a * rcp_(b); }

// 1/sqrt(x), lane by lane the scalar rsqrt_ (one Newton step from the
// hardware approximation, residual by TwoProd and FMA).
__device__ __forceinline__ dw2 rsqrt_(dw2 x) {
  const float2 y0 = make_float2(dw_rsqrt_approx(x.hi.x), dw_rsqrt_approx(x.hi.y));
  const float2 q = p_mul(y0, y0);
  const float2 qe = p_fma(y0, y0, p_neg(q));
  float2 m = p_fma(x.hi, q, make_float2(-1.0f, -1.0f));
  m = p_fma(x.hi, qe, m);
  m = p_fma(x.lo, q, m);
  const float2 c = p_fma(make_float2(0.375f, 0.375f), m, make_float2(-0.5f, -0.5f));
  dw2 z;
  dw2_fast_two_sum(y0, p_mul(y0, p_mul(m, c)), z.hi, z.lo);
  return z;
}

// sqrt(x) = x / sqrt(x), exactly 0 in a lane whose x is 0 (as the scalar sqrt_).
__device__ __forceinline__ dw2 sqrt_(dw2 x) {
  const dw2 r = x * rsqrt_(x);
  const bool zx = x.hi.x == 0.0f, zy = x.hi.y == 0.0f;
  return dw2(make_float2(zx ? 0.0f : r.hi.x, zy ? 0.0f : r.hi.y), make_float2(zx ? 0.0f : r.lo.x, zy ? 0.0f : r.lo.y));
}

__device__ __forceinline__ dw2 abs_(dw2 x) {
  const float sx = x.hi.x < 0.0f ? -1.0f : 1.0f, sy = x.hi.y < 0.0f ? -1.0f : 1.0f;
  const float2 s = make_float2(sx, sy);
  return dw2(p_mul(s, x.hi), p_mul(s, x.lo));
}

// Lanes and their assembly.
__device__ __forceinline__ dw lane_x(dw2 v) { return dw(v.hi.x, v.lo.x); }
__device__ __forceinline__ dw lane_y(dw2 v) { return dw(v.hi.y, v.lo.y); }
__device__ __forceinline__ dw2 pack2(dw a, dw b) { return dw2(make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)); }
__device__ __forceinline__ dw2 splat2(dw a) { return pack2(a, a); }

// Range guard of packed values: both lanes.
struct DwGuard2 : DwGuard {
  using DwGuard::check;
  __device__ __forceinline__ void check(dw2 x) {
    check(lane_x(x));
    check(lane_y(x));
  }
};

// Two doubles (one per lane) to and from packed double-word, lane by lane the
// scalar conversions.
template <DwConv C = DwConv::kClamp>
__device__ __forceinline__ dw2 dw2_from_double2(double2 x, DwGuard& g) {
  return pack2(dw_from_double<C>(x.x, g), dw_from_double<C>(x.y, g));
}
template <DwConv C = DwConv::kClamp>
__device__ __forceinline__ double2 dw2_to_double2(dw2 x) {
  return make_double2(dw_to_double<C>(lane_x(x)), dw_to_double<C>(lane_y(x)));
}

// x^y of each lane through FP64 (the optional entropy output only).
__device__ __forceinline__ dw2 pow_(dw2 x, dw2 y) {
  return pack2(pow_(lane_x(x), lane_x(y)), pow_(lane_y(x), lane_y(y)));
}

}  // namespace fdbb
