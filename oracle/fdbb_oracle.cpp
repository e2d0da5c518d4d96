// fdbb_oracle.cpp -- plain FP64 CPU oracle for the compressible-Euler building
// blocks of FDBB (Moeller & Jaeschke, "FDBB: Fluid Dynamics Building Blocks").
//
// TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
// path.  Only the test suite, the smoke check and the CPU-baseline leg of the
// benchmark may load it.  The product library never links, loads or calls it,
// and this file shares no code, header or constant table with the CUDA path.
//
// Every formula is written out from its definition, point by point, in plain
// IEEE double arithmetic (compile with -O2 -ffp-contract=off so that no FMA
// contraction changes the rounding).  Nothing is fused, blocked or reordered.
//
// Notation (paper, section 2.2, "Variables" and "Inviscid Fluxes"):
//   dimension D in {1,2,3}, nv = D + 2 state components per point,
//   conservative U = (rho, m_1..m_D, rhoE) with m = rho v,
//   primitive    V = (rho, v_1..v_D, p),
//   ideal gas with adiabatic index gamma = c_p / c_v (1.4 in the paper).
// Fields are structure-of-arrays: component k of all n points is one
// contiguous array ("plane"); the caller passes an array of plane pointers.
//
// Formulas the paper names but does not print (flux Jacobians, eigenvectors,
// characteristic variables, Riemann invariants) are the standard ideal-gas
// Euler algebra (e.g. E. F. Toro, "Riemann Solvers and Numerical Methods for
// Fluid Dynamics", 3rd ed., sections 3.1-3.2).
//
// Tolerance scale.  Each formula is a template over the number type.  With
// T = double it is the oracle.  With T = Err the same formula propagates a
// first-order running-error bound S (Wilkinson): if every input is exact and
// every operation rounds with unit roundoff u, the computed value differs
// from the exact one by at most about u * S.  A GPU result g is accepted when
// |g - o| <= tol * S.  S >= |o|, and S is much larger than |o| exactly where
// the formula cancels (e.g. rhoE - rho q at high Mach), which is where a
// different but equally valid evaluation order legitimately differs.
//
// Parity pins: see the oracle self-tests (tests/test_oracle_pins.py); no
// function in this file is left unpinned.

#include <cmath>
#include <cstdint>
#include <cstddef>

namespace {

// ---------------------------------------------------------------------------
// Number types
// ---------------------------------------------------------------------------

// Value plus first-order running-error scale.
struct Err {
  double v;  // value, computed exactly as the double oracle computes it
  double s;  // error scale: |computed - exact| <~ u * s
};

inline Err operator+(Err a, Err b) {
  double v = a.v + b.v;
  return {v, std::fabs(v) + a.s + b.s};
}
inline Err operator-(Err a, Err b) {
  double v = a.v - b.v;
  return {v, std::fabs(v) + a.s + b.s};
}
inline Err operator-(Err a) { return {-a.v, a.s}; }
inline Err operator*(Err a, Err b) {
  double v = a.v * b.v;
  return {v, std::fabs(v) + a.s * std::fabs(b.v) + std::fabs(a.v) * b.s};
}
inline Err operator/(Err a, Err b) {
  double v = a.v / b.v;
  return {v, std::fabs(v) + (a.s + std::fabs(v) * b.s) / std::fabs(b.v)};
}
inline Err sqrt_(Err a) {
  double v = std::sqrt(a.v);
  // d sqrt(x) = dx / (2 sqrt(x)); at x == 0 the bound is sqrt(u s)/u, which
  // is finite and large, as it should be.
  double prop = (v > 0.0) ? a.s / (2.0 * v) : std::sqrt(a.s / 0x1p-53);
  return {v, v + prop};
}
inline double sqrt_(double a) { return std::sqrt(a); }
inline double abs_(double a) { return std::fabs(a); }
inline Err abs_(Err a) { return {std::fabs(a.v), a.s}; }

// x^y for x > 0 (entropy p / rho^gamma); libm pow is within about 1 ulp.
inline double pow_(double x, double y) { return std::pow(x, y); }
inline Err pow_(Err x, Err y) {
  double v = std::pow(x.v, y.v);
  double rel = 2.0 + (x.v != 0.0 ? std::fabs(y.v) * x.s / std::fabs(x.v) : 0.0);
  return {v, std::fabs(v) * rel};
}

template <class T> inline T lit(double x);
template <> inline double lit<double>(double x) { return x; }
template <> inline Err lit<Err>(double x) { return {x, 0.0}; }  // exact input

inline double val(double x) { return x; }
inline double val(Err x) { return x.v; }
inline double scl(double x) { return std::fabs(x); }
inline double scl(Err x) { return x.s; }

// ---------------------------------------------------------------------------
// Point-wise formulas
// ---------------------------------------------------------------------------

// Conservative state of one point and the secondary variables derived from
// it (paper section 2.2, "Variables": pressure from U for a perfect gas with
// gamma = c_p / c_v; Fig. 7 computes p from (rho, m_x, m_y, m_z, rhoE)).
template <class T> struct State {
  int D;
  T gamma, a1;        // gamma and a1 = gamma - 1
  T rho, m[3], rhoE;  // conservative variables
  T v[3];             // velocity v_i = m_i / rho
  T q;                // kinetic energy per unit mass, q = |v|^2 / 2
  T p;                // pressure p = (gamma - 1) (rhoE - rho q)
  T c;                // speed of sound c = sqrt(gamma p / rho)
  T H;                // total specific enthalpy H = (rhoE + p) / rho
  // Set only by the general-EOS state (state_from_cons_eos):
  T e;                // specific internal energy
  T dp[5];            // dp/dU: dp/drho, dp/dm_1..dp/dm_D, dp/drhoE (others unused)
};

template <class T>
State<T> state_from_cons(int D, double gamma, const double* const* U, int64_t i) {
  State<T> s;
  s.D = D;
  s.gamma = lit<T>(gamma);
  s.a1 = s.gamma - lit<T>(1.0);
  s.rho = lit<T>(U[0][i]);
  for (int k = 0; k < 3; ++k) s.m[k] = lit<T>(0.0);
  for (int k = 0; k < D; ++k) s.m[k] = lit<T>(U[1 + k][i]);
  s.rhoE = lit<T>(U[D + 1][i]);
  for (int k = 0; k < 3; ++k) s.v[k] = lit<T>(0.0);
  for (int k = 0; k < D; ++k) s.v[k] = s.m[k] / s.rho;
  T v2 = s.v[0] * s.v[0];
  for (int k = 1; k < D; ++k) v2 = v2 + s.v[k] * s.v[k];
  s.q = lit<T>(0.5) * v2;
  s.p = s.a1 * (s.rhoE - s.rho * s.q);
  s.c = sqrt_(s.gamma * s.p / s.rho);
  s.H = (s.rhoE + s.p) / s.rho;
  return s;
}

// Inviscid flux in direction d (paper section 2.2, "Inviscid Fluxes": the
// N_U x N_D flux tensor F(U) = [rho v; rho v (x) v + I p; v (rhoE + p)];
// column d of that tensor):
//   F_d[0]     = m_d
//   F_d[1+i]   = m_d v_i + delta_{id} p
//   F_d[nv-1]  = v_d (rhoE + p)
template <class T> void flux_d(const State<T>& s, int d, T* F) {
  const int D = s.D;
  F[0] = s.m[d];
  for (int i = 0; i < D; ++i) {
    F[1 + i] = s.m[d] * s.v[i];
    if (i == d) F[1 + i] = F[1 + i] + s.p;
  }
  F[D + 1] = s.v[d] * (s.rhoE + s.p);
}

// Flux Jacobian A_d = dF_d / dU, row-major A[r*nv + col], rows and columns in
// U order (the paper names the flux Jacobians in section 1 and Fig. 1; the
// entries are the derivative of the flux above with p = a1 (rhoE - |m|^2/(2 rho)),
// dp/drho = a1 q, dp/dm_j = -a1 v_j, dp/drhoE = a1).  With phi = a1 q, u = v_d:
//   row 0     : e_{1+d}
//   row 1+i   : (-u v_i, v_i at col 1+d, u at col 1+i)            (i != d)
//   row 1+d   : (phi - u^2, -a1 v_j at col 1+j (j != d), (3 - gamma) u at
//                col 1+d, a1 at col nv-1)
//   row nv-1  : (u (phi - H), -a1 u v_j at col 1+j (j != d),
//                H - a1 u^2 at col 1+d, gamma u at col nv-1)
template <class T> void jacobian_d(const State<T>& s, int d, T* A) {
  const int D = s.D, nv = D + 2;
  const T zero = lit<T>(0.0), one = lit<T>(1.0);
  for (int k = 0; k < nv * nv; ++k) A[k] = zero;
  const T u = s.v[d];
  const T phi = s.a1 * s.q;
  A[0 * nv + (1 + d)] = one;
  for (int i = 0; i < D; ++i) {
    T* row = A + (1 + i) * nv;
    if (i != d) {
      row[0] = -(u * s.v[i]);
      row[1 + d] = s.v[i];
      row[1 + i] = u;
    } else {
      row[0] = phi - u * u;
      for (int j = 0; j < D; ++j)
        if (j != d) row[1 + j] = -(s.a1 * s.v[j]);
      row[1 + d] = (lit<T>(3.0) - s.gamma) * u;
      row[nv - 1] = s.a1;
    }
  }
  T* last = A + (nv - 1) * nv;
  last[0] = u * (phi - s.H);
  for (int j = 0; j < D; ++j)
    if (j != d) last[1 + j] = -(s.a1 * u * s.v[j]);
  last[1 + d] = s.H - s.a1 * u * u;
  last[nv - 1] = s.gamma * u;
}

// Tangential directions of d in ascending order (for the shear waves).
inline int tangential(int D, int d, int k) {
  int t = -1;
  for (int j = 0, cnt = 0; j < D; ++j)
    if (j != d) {
      if (cnt == k) t = j;
      ++cnt;
    }
  return t;
}

// Right eigenvectors of A_d as the columns of R (row-major R[r*nv + k]),
// eigenvalues lambda = (u - c, u, ..., u, u + c):
//   r_1        = (1, v - c e_d, H - u c)
//   r_2        = (1, v, q)
//   r_{2+k}    = (0, e_t, v_t)      t = k-th tangential direction
//   r_nv       = (1, v + c e_d, H + u c)
template <class T> void right_eig_d(const State<T>& s, int d, T* R, T* lam) {
  const int D = s.D, nv = D + 2;
  const T zero = lit<T>(0.0), one = lit<T>(1.0);
  const T u = s.v[d], c = s.c;
  for (int k = 0; k < nv * nv; ++k) R[k] = zero;
  // column 0: acoustic wave u - c
  R[0 * nv + 0] = one;
  for (int i = 0; i < D; ++i) R[(1 + i) * nv + 0] = (i == d) ? s.v[i] - c : s.v[i];
  R[(nv - 1) * nv + 0] = s.H - u * c;
  // column 1: entropy wave
  R[0 * nv + 1] = one;
  for (int i = 0; i < D; ++i) R[(1 + i) * nv + 1] = s.v[i];
  R[(nv - 1) * nv + 1] = s.q;
  // columns 2 .. nv-2: shear waves
  for (int k = 0; k < D - 1; ++k) {
    int t = tangential(D, d, k);
    R[(1 + t) * nv + (2 + k)] = one;
    R[(nv - 1) * nv + (2 + k)] = s.v[t];
  }
  // column nv-1: acoustic wave u + c
  R[0 * nv + (nv - 1)] = one;
  for (int i = 0; i < D; ++i) R[(1 + i) * nv + (nv - 1)] = (i == d) ? s.v[i] + c : s.v[i];
  R[(nv - 1) * nv + (nv - 1)] = s.H + u * c;
  if (lam) {
    lam[0] = u - c;
    for (int k = 1; k < nv - 1; ++k) lam[k] = u;
    lam[nv - 1] = u + c;
  }
}

// Left eigenvectors of A_d as the rows of L = R^{-1}, with b1 = a1 / c^2 and
// b2 = q b1 (v written in component slots 1..D):
//   l_1     = 1/2 (b2 + u/c, -b1 v - e_d / c, b1)
//   l_2     = (1 - b2, b1 v, -b1)
//   l_{2+k} = (-v_t, e_t, 0)
//   l_nv    = 1/2 (b2 - u/c, -b1 v + e_d / c, b1)
template <class T> void left_eig_d(const State<T>& s, int d, T* L) {
  const int D = s.D, nv = D + 2;
  const T zero = lit<T>(0.0), one = lit<T>(1.0), half = lit<T>(0.5);
  const T u = s.v[d], c = s.c;
  const T b1 = s.a1 / (c * c);
  const T b2 = s.q * b1;
  for (int k = 0; k < nv * nv; ++k) L[k] = zero;
  T* l1 = L + 0 * nv;
  T* l2 = L + 1 * nv;
  T* ln = L + (nv - 1) * nv;
  l1[0] = half * (b2 + u / c);
  ln[0] = half * (b2 - u / c);
  l2[0] = one - b2;
  for (int i = 0; i < D; ++i) {
    T bv = b1 * s.v[i];
    if (i == d) {
      l1[1 + i] = half * (-bv - one / c);
      ln[1 + i] = half * (-bv + one / c);
    } else {
      l1[1 + i] = half * (-bv);
      ln[1 + i] = half * (-bv);
    }
    l2[1 + i] = bv;
  }
  l1[nv - 1] = half * b1;
  ln[nv - 1] = half * b1;
  l2[nv - 1] = -b1;
  for (int k = 0; k < D - 1; ++k) {
    int t = tangential(D, d, k);
    T* lk = L + (2 + k) * nv;
    lk[0] = -s.v[t];
    lk[1 + t] = one;
  }
}

// y = M x for an nv x nv row-major matrix, summed left to right.
template <class T> void matvec(int nv, const T* M, const T* x, T* y) {
  for (int r = 0; r < nv; ++r) {
    T acc = M[r * nv + 0] * x[0];
    for (int k = 1; k < nv; ++k) acc = acc + M[r * nv + k] * x[k];
    y[r] = acc;
  }
}

// y = M^T x.
template <class T> void matvec_t(int nv, const T* M, const T* x, T* y) {
  for (int col = 0; col < nv; ++col) {
    T acc = M[0 * nv + col] * x[0];
    for (int r = 1; r < nv; ++r) acc = acc + M[r * nv + col] * x[r];
    y[col] = acc;
  }
}

// Primitive-variable forms (paper section 2.2, Fig. 9: Variables<eos, dim,
// EnumForm::primitive>, V = (rho, v, p)).
//   Flux from V: F_d = (rho u, rho u v + p e_d, u (gamma/(gamma-1) p + rho |v|^2/2)),
//   u = v_d (the same physical flux, written in V).
template <class T> void flux_prim_d(int D, double g, const double* const* V, int64_t i, int d, T* F) {
  const T gamma = lit<T>(g), a1 = gamma - lit<T>(1.0);
  const T rho = lit<T>(V[0][i]), p = lit<T>(V[D + 1][i]);
  T v[3];
  for (int k = 0; k < D; ++k) v[k] = lit<T>(V[1 + k][i]);
  T v2 = v[0] * v[0];
  for (int k = 1; k < D; ++k) v2 = v2 + v[k] * v[k];
  const T u = v[d];
  F[0] = rho * u;
  for (int k = 0; k < D; ++k) {
    F[1 + k] = rho * u * v[k];
    if (k == d) F[1 + k] = F[1 + k] + p;
  }
  F[D + 1] = u * (gamma / a1 * p + lit<T>(0.5) * rho * v2);
}

// Jacobian of that flux with respect to V, B_d = dF_d/dV (row-major, rows in
// U order, columns in V order), from differentiating the formula above:
//   row 0    : (u, rho at col 1+d, 0)
//   row 1+i  : (u v_i, rho (delta_jd v_i + delta_ij u) at col 1+j, delta_id at col nv-1)
//   row nv-1 : (u |v|^2/2, delta_jd (gamma/(gamma-1) p + rho |v|^2/2) + rho u v_j at col 1+j,
//               gamma/(gamma-1) u at col nv-1)
template <class T> void jac_prim_d(int D, double g, const double* const* V, int64_t i, int d, T* B) {
  const int nv = D + 2;
  const T gamma = lit<T>(g), a1 = gamma - lit<T>(1.0), zero = lit<T>(0.0), one = lit<T>(1.0);
  const T rho = lit<T>(V[0][i]), p = lit<T>(V[D + 1][i]);
  T v[3];
  for (int k = 0; k < D; ++k) v[k] = lit<T>(V[1 + k][i]);
  T v2 = v[0] * v[0];
  for (int k = 1; k < D; ++k) v2 = v2 + v[k] * v[k];
  const T u = v[d];
  for (int k = 0; k < nv * nv; ++k) B[k] = zero;
  B[0] = u;
  B[1 + d] = rho;
  for (int r = 0; r < D; ++r) {
    T* row = B + (1 + r) * nv;
    row[0] = u * v[r];
    for (int j = 0; j < D; ++j) {
      T e = zero;
      if (j == d) e = e + rho * v[r];
      if (j == r) e = e + rho * u;
      row[1 + j] = e;
    }
    row[nv - 1] = (r == d) ? one : zero;
  }
  T* last = B + (nv - 1) * nv;
  last[0] = lit<T>(0.5) * u * v2;
  for (int j = 0; j < D; ++j) {
    T e = rho * u * v[j];
    if (j == d) e = e + (gamma / a1 * p + lit<T>(0.5) * rho * v2);
    last[1 + j] = e;
  }
  last[nv - 1] = gamma / a1 * u;
}

// Roe-averaged state between left and right states (P. L. Roe, J. Comput.
// Phys. 43, 1981; Toro ch. 11): with w = sqrt(rho),
//   v^ = (w_L v_L + w_R v_R) / (w_L + w_R),  H^ = (w_L H_L + w_R H_R) / (w_L + w_R),
//   q^ = |v^|^2 / 2,  c^ = sqrt((gamma - 1)(H^ - q^)).
// Only the fields the eigenvectors use (v, q, H, c, gamma, a1) are set.
template <class T> State<T> roe_state(const State<T>& L, const State<T>& R) {
  State<T> s = L;
  const T wL = sqrt_(L.rho), wR = sqrt_(R.rho);
  const T den = wL + wR;
  for (int i = 0; i < L.D; ++i) s.v[i] = (wL * L.v[i] + wR * R.v[i]) / den;
  s.H = (wL * L.H + wR * R.H) / den;
  T v2 = s.v[0] * s.v[0];
  for (int i = 1; i < L.D; ++i) v2 = v2 + s.v[i] * s.v[i];
  s.q = lit<T>(0.5) * v2;
  s.c = sqrt_(s.a1 * (s.H - s.q));
  return s;
}

// Roe flux in direction d: Fh = (F_d(U_L) + F_d(U_R))/2 - 1/2 sum_k |lambda^_k|
// alpha_k r^_k with alpha = L^ (U_R - U_L), all at the Roe state.
template <class T> void roe_flux_d(const State<T>& L, const State<T>& R, int d, T* Fh) {
  const int D = L.D, nv = D + 2;
  T fL[5], fR[5], Rm[25], Lm[25], lam[5], dU[5], alpha[5];
  flux_d(L, d, fL);
  flux_d(R, d, fR);
  const State<T> s = roe_state(L, R);
  right_eig_d(s, d, Rm, lam);
  left_eig_d(s, d, Lm);
  dU[0] = R.rho - L.rho;
  for (int i = 0; i < D; ++i) dU[1 + i] = R.m[i] - L.m[i];
  dU[nv - 1] = R.rhoE - L.rhoE;
  matvec(nv, Lm, dU, alpha);
  for (int q = 0; q < nv; ++q) {
    T diss = abs_(lam[0]) * alpha[0] * Rm[q * nv + 0];
    for (int k = 1; k < nv; ++k) diss = diss + abs_(lam[k]) * alpha[k] * Rm[q * nv + k];
    Fh[q] = lit<T>(0.5) * (fL[q] + fR[q]) - lit<T>(0.5) * diss;
  }
}

// ---------------------------------------------------------------------------
// Plane output helpers
// ---------------------------------------------------------------------------

template <class T>
inline void put(double* const* out, double* const* scale, int k, int64_t i, T x) {
  if (out && out[k]) out[k][i] = val(x);
  if (scale && scale[k]) scale[k][i] = scl(x);
}

inline bool bad_dim(int D) { return D < 1 || D > 3; }

// ---------------------------------------------------------------------------
// Array drivers, one per building block.  Each loops over points and calls
// the point-wise formula above.  `scale` (may be NULL) receives the error
// scale S of every written output.
// ---------------------------------------------------------------------------

template <class T>
void run_v_mag2(int D, int64_t n, const double* const* U, double* const* out, double* const* sc) {
  // Paper section 3, Eq. (2): y <- (m_x.*m_x + m_y.*m_y + m_z.*m_z) ./ (rho.*rho)
  for (int64_t i = 0; i < n; ++i) {
    T rho = lit<T>(U[0][i]);
    T m = lit<T>(U[1][i]);
    T num = m * m;
    for (int k = 1; k < D; ++k) {
      T mk = lit<T>(U[1 + k][i]);
      num = num + mk * mk;
    }
    put(out, sc, 0, i, num / (rho * rho));
  }
}

template <class T>
void run_prim_from_cons(int D, double g, int64_t n, const double* const* U, double* const* V,
                        double* const* sc) {
  // Paper section 2.2, Fig. 9: V = varU::primitive(U), V = (rho, v, p).
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    put(V, sc, 0, i, s.rho);
    for (int k = 0; k < D; ++k) put(V, sc, 1 + k, i, s.v[k]);
    put(V, sc, D + 1, i, s.p);
  }
}

template <class T>
void run_cons_from_prim(int D, double g, int64_t n, const double* const* V, double* const* U,
                        double* const* sc) {
  // Paper section 2.2, Fig. 9: U = varV::conservative(V):
  //   m_i = rho v_i, rhoE = p / (gamma - 1) + rho |v|^2 / 2.
  for (int64_t i = 0; i < n; ++i) {
    T gamma = lit<T>(g);
    T a1 = gamma - lit<T>(1.0);
    T rho = lit<T>(V[0][i]);
    T v2 = lit<T>(0.0);
    put(U, sc, 0, i, rho);
    for (int k = 0; k < D; ++k) {
      T vk = lit<T>(V[1 + k][i]);
      put(U, sc, 1 + k, i, rho * vk);
      v2 = (k == 0) ? vk * vk : v2 + vk * vk;
    }
    T p = lit<T>(V[D + 1][i]);
    put(U, sc, D + 1, i, p / a1 + lit<T>(0.5) * rho * v2);
  }
}

template <class T>
void run_eos(int D, double g, int64_t n, const double* const* U, double* const* out,
             double* const* sc) {
  // Paper section 2.2, "Variables" and "Equations of state": ideal gas
  // p = (gamma - 1) rho e; speed of sound c = sqrt(gamma p / rho).
  // out = {p, c}.
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    put(out, sc, 0, i, s.p);
    put(out, sc, 1, i, s.c);
  }
}

template <class T>
void run_riemann(int D, int d, double g, int64_t n, const double* const* U, double* const* out,
                 double* const* sc) {
  // Riemann invariants along direction d (paper section 1 names them):
  //   w- = u - 2 c / (gamma - 1),  w+ = u + 2 c / (gamma - 1),  u = v_d,
  // and the entropy s = p / rho^gamma.  out = {w-, w+, s}.
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    T twoc = lit<T>(2.0) * s.c / s.a1;
    put(out, sc, 0, i, s.v[d] - twoc);
    put(out, sc, 1, i, s.v[d] + twoc);
    put(out, sc, 2, i, s.p / pow_(s.rho, s.gamma));
  }
}

template <class T>
void run_flux(int D, int dir, double g, int64_t n, const double* const* U, double* const* F,
              double* const* sc) {
  // dir in [0, D): one flux column (nv planes); dir == -1: all columns,
  // direction-major, plane d*nv + k.
  const int nv = D + 2;
  T f[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    for (int d = 0; d < D; ++d) {
      if (dir >= 0 && d != dir) continue;
      flux_d(s, d, f);
      int base = (dir < 0) ? d * nv : 0;
      for (int k = 0; k < nv; ++k) put(F, sc, base + k, i, f[k]);
    }
  }
}

template <class T>
void run_flux_jac(int D, int d, double g, int64_t n, const double* const* U, double* const* A,
                  double* const* sc) {
  const int nv = D + 2;
  T a[25];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    jacobian_d(s, d, a);
    for (int k = 0; k < nv * nv; ++k) put(A, sc, k, i, a[k]);
  }
}

template <class T>
void run_char(int D, int d, double g, int inverse, int64_t n, const double* const* U,
              const double* const* W, double* const* Y, double* const* sc) {
  // Characteristic transform at the local state (paper section 1 names
  // characteristic variables): forward Y = L_d(U) W, inverse Y = R_d(U) W.
  const int nv = D + 2;
  T M[25], w[5], y[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    if (inverse)
      right_eig_d(s, d, M, (T*)nullptr);
    else
      left_eig_d(s, d, M);
    for (int k = 0; k < nv; ++k) w[k] = lit<T>(W[k][i]);
    matvec(nv, M, w, y);
    for (int k = 0; k < nv; ++k) put(Y, sc, k, i, y[k]);
  }
}

template <class T>
void run_flux_vjp(int D, int d, double g, int64_t n, const double* const* U, const double* const* G,
                  double* const* gU, double* const* sc) {
  // Vector-Jacobian product of the direction-d flux: gU = A_d(U)^T G.
  const int nv = D + 2;
  T a[25], gg[5], y[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    jacobian_d(s, d, a);
    for (int k = 0; k < nv; ++k) gg[k] = lit<T>(G[k][i]);
    matvec_t(nv, a, gg, y);
    for (int k = 0; k < nv; ++k) put(gU, sc, k, i, y[k]);
  }
}

template <class T>
void run_fused(int D, int dj, double g, int64_t n, const double* const* U, const double* const* W,
               double* const* out, double* const* sc) {
  // All fluxes F_0..F_{D-1} (planes d*nv + k), then A_dj (nv*nv planes), then
  // Y = L_dj(U) W (nv planes): exactly run_flux(dir=-1), run_flux_jac and
  // run_char(forward) one after the other.
  const int nv = D + 2;
  const int off_A = D * nv, off_Y = D * nv + nv * nv;
  T f[5], a[25], M[25], w[5], y[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    for (int d = 0; d < D; ++d) {
      flux_d(s, d, f);
      for (int k = 0; k < nv; ++k) put(out, sc, d * nv + k, i, f[k]);
    }
    jacobian_d(s, dj, a);
    for (int k = 0; k < nv * nv; ++k) put(out, sc, off_A + k, i, a[k]);
    left_eig_d(s, dj, M);
    for (int k = 0; k < nv; ++k) w[k] = lit<T>(W[k][i]);
    matvec(nv, M, w, y);
    for (int k = 0; k < nv; ++k) put(out, sc, off_Y + k, i, y[k]);
  }
}

template <class T>
void run_flux_prim(int D, int dir, double g, int64_t n, const double* const* V, double* const* F,
                   double* const* sc) {
  const int nv = D + 2;
  T f[5];
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < D; ++d) {
      if (dir >= 0 && d != dir) continue;
      flux_prim_d<T>(D, g, V, i, d, f);
      const int base = (dir < 0) ? d * nv : 0;
      for (int k = 0; k < nv; ++k) put(F, sc, base + k, i, f[k]);
    }
}

template <class T>
void run_jac_prim(int D, int d, double g, int64_t n, const double* const* V, double* const* B,
                  double* const* sc) {
  const int nv = D + 2;
  T b[25];
  for (int64_t i = 0; i < n; ++i) {
    jac_prim_d<T>(D, g, V, i, d, b);
    for (int k = 0; k < nv * nv; ++k) put(B, sc, k, i, b[k]);
  }
}

template <class T>
void run_temperature(int D, double g, double cv, int64_t n, const double* const* U, double* const* out,
                     double* const* sc) {
  // Temperature of the perfect gas from (rho, e) (paper section 2.2,
  // "Equations of state", the T_rhoe member of the EOS prototype, Fig. 10):
  // T = e / c_v, e = (rhoE - rho q) / rho.
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons<T>(D, g, U, i);
    const T e = (s.rhoE - s.rho * s.q) / s.rho;
    put(out, sc, 0, i, e / lit<T>(cv));
  }
}

template <class T>
void run_roe_flux(int D, int d, double g, int64_t n, const double* const* UL, const double* const* UR,
                  double* const* F, double* const* sc) {
  // Roe flux between the states UL and UR of each point (direction d).
  const int nv = D + 2;
  T f[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> L = state_from_cons<T>(D, g, UL, i);
    State<T> R = state_from_cons<T>(D, g, UR, i);
    roe_flux_d(L, R, d, f);
    for (int k = 0; k < nv; ++k) put(F, sc, k, i, f[k]);
  }
}

template <class T>
void run_roe_char(int D, int d, double g, int inverse, int64_t n, const double* const* UL,
                  const double* const* UR, const double* const* W, double* const* Y, double* const* sc) {
  // Characteristic transform at the Roe-averaged state of (UL, UR):
  // forward Y = L^ W, inverse Y = R^ W.
  const int nv = D + 2;
  T M[25], w[5], y[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> L = state_from_cons<T>(D, g, UL, i);
    State<T> R = state_from_cons<T>(D, g, UR, i);
    const State<T> s = roe_state(L, R);
    if (inverse)
      right_eig_d(s, d, M, (T*)nullptr);
    else
      left_eig_d(s, d, M);
    for (int k = 0; k < nv; ++k) w[k] = lit<T>(W[k][i]);
    matvec(nv, M, w, y);
    for (int k = 0; k < nv; ++k) put(Y, sc, k, i, y[k]);
  }
}

// ---------------------------------------------------------------------------
// General equations of state (paper section 2.2, "Equations of state": a
// user EOS of the form f(p, V, T) = 0 supplies p(rho, e) and T(rho, e),
// Fig. 10).  The paper prints no EOS besides the ideal gas; two standard
// families stand in for user EOS here:
//
//  NASG, the Noble-Abel stiffened gas (O. Le Metayer and R. Saurel, Phys.
//  Fluids 28, 046102, 2016), parameters gamma, p_inf, b, q, c_v:
//     p(rho, e)   = (gamma - 1)(e - q) rho / (1 - b rho) - gamma p_inf
//     T(rho, e)   = (e - q - p_inf (1/rho - b)) / c_v
//     rho e(rho,p) = (p + gamma p_inf)(1 - b rho)/(gamma - 1) + rho q
//  (the ideal gas for p_inf = b = q = 0, the stiffened gas for b = 0);
//
//  van der Waals with caloric law e = c_v T - a rho, parameters gamma, a, b, c_v:
//     p(rho, e)   = (gamma - 1)(rho e + a rho^2)/(1 - b rho) - a rho^2
//     T(rho, e)   = (e + a rho) / c_v
//     rho e(rho,p) = (p + a rho^2)(1 - b rho)/(gamma - 1) - a rho^2.
//
// The partial derivatives p_rho = dp/drho at constant e, p_e = dp/de at
// constant rho, and those of rho e(rho, p) are written out by hand below.
// Everything else follows from the definitions:
//   speed of sound  c^2 = dp/drho at constant entropy = p_rho + p_e p / rho^2
//   (de = p / rho^2 drho along an isentrope), and the Euler algebra of the
//   ideal-gas functions above with the pressure gradient dp/dU in place of
//   the ideal-gas one.
// ---------------------------------------------------------------------------

enum { EOS_NASG = 1, EOS_VDW = 2 };

struct EosModel {
  int kind;
  double gamma, p_inf, b, q, a, cv;
};

// params = {kind, gamma, p_inf, b, q, a, cv}
inline bool eos_from_params(const double* prm, EosModel& M) {
  if (!prm) return false;
  M.kind = (int)prm[0];
  M.gamma = prm[1];
  M.p_inf = prm[2];
  M.b = prm[3];
  M.q = prm[4];
  M.a = prm[5];
  M.cv = prm[6];
  if (M.kind != EOS_NASG && M.kind != EOS_VDW) return false;
  if (!(M.gamma > 1.0) || !(M.cv > 0.0) || !(M.b >= 0.0)) return false;
  if (M.kind == EOS_NASG && !(M.p_inf >= 0.0)) return false;
  if (M.kind == EOS_VDW && !(M.a >= 0.0)) return false;
  return true;
}

// p, p_rho = dp/drho|_e and p_e = dp/de|_rho at (rho, e).
template <class T> void eos_p(const EosModel& M, T rho, T e, T& p, T& p_rho, T& p_e) {
  const T g = lit<T>(M.gamma), a1 = g - lit<T>(1.0), one = lit<T>(1.0);
  const T b = lit<T>(M.b);
  const T den = one - b * rho;  // 1 - b rho
  if (M.kind == EOS_NASG) {
    const T q = lit<T>(M.q), pinf = lit<T>(M.p_inf);
    // d/drho [rho / (1 - b rho)] = 1 / (1 - b rho)^2
    p = a1 * (e - q) * rho / den - g * pinf;
    p_rho = a1 * (e - q) / (den * den);
    p_e = a1 * rho / den;
  } else {
    const T a = lit<T>(M.a);
    const T num = rho * e + a * rho * rho;  // rho e + a rho^2
    p = a1 * num / den - a * rho * rho;
    // d/drho [num / den] = ((e + 2 a rho) den + b num) / den^2
    p_rho = a1 * ((e + lit<T>(2.0) * a * rho) * den + b * num) / (den * den) - lit<T>(2.0) * a * rho;
    p_e = a1 * rho / den;
  }
}

// Temperature T(rho, e).
template <class T> T eos_T(const EosModel& M, T rho, T e) {
  const T cv = lit<T>(M.cv);
  if (M.kind == EOS_NASG) {
    const T one = lit<T>(1.0);
    return (e - lit<T>(M.q) - lit<T>(M.p_inf) * (one / rho - lit<T>(M.b))) / cv;
  }
  return (e + lit<T>(M.a) * rho) / cv;
}

// Internal energy density rho e(rho, p) and its partial derivatives
// z_rho = d(rho e)/drho|_p, z_p = d(rho e)/dp|_rho.
template <class T> void eos_rhoe(const EosModel& M, T rho, T p, T& z, T& z_rho, T& z_p) {
  const T g = lit<T>(M.gamma), a1 = g - lit<T>(1.0), one = lit<T>(1.0);
  const T b = lit<T>(M.b);
  const T den = one - b * rho;
  if (M.kind == EOS_NASG) {
    const T q = lit<T>(M.q), pinf = lit<T>(M.p_inf);
    const T pp = p + g * pinf;
    z = pp * den / a1 + rho * q;
    z_rho = q - b * pp / a1;
    z_p = den / a1;
  } else {
    const T a = lit<T>(M.a);
    const T pp = p + a * rho * rho;
    z = pp * den / a1 - a * rho * rho;
    // d/drho: (2 a rho (1 - b rho) - b (p + a rho^2)) / (gamma - 1) - 2 a rho
    z_rho = (lit<T>(2.0) * a * rho * den - b * pp) / a1 - lit<T>(2.0) * a * rho;
    z_p = den / a1;
  }
}

// Conservative state under a general EOS: e = (rhoE - rho q)/rho, p and c as
// above, H = (rhoE + p)/rho and the pressure gradient dp/dU by the chain rule
// through e(rho, m, rhoE):
//   de/drho = (q - e)/rho,  de/dm_j = -v_j/rho,  de/drhoE = 1/rho, so
//   dp/drho = p_rho + p_e (q - e)/rho, dp/dm_j = -p_e v_j/rho, dp/drhoE = p_e/rho.
template <class T>
State<T> state_from_cons_eos(int D, const EosModel& M, const double* const* U, int64_t i) {
  State<T> s;
  s.D = D;
  s.gamma = lit<T>(M.gamma);
  s.a1 = s.gamma - lit<T>(1.0);
  s.rho = lit<T>(U[0][i]);
  for (int k = 0; k < 3; ++k) s.m[k] = lit<T>(0.0);
  for (int k = 0; k < D; ++k) s.m[k] = lit<T>(U[1 + k][i]);
  s.rhoE = lit<T>(U[D + 1][i]);
  for (int k = 0; k < 3; ++k) s.v[k] = lit<T>(0.0);
  for (int k = 0; k < D; ++k) s.v[k] = s.m[k] / s.rho;
  T v2 = s.v[0] * s.v[0];
  for (int k = 1; k < D; ++k) v2 = v2 + s.v[k] * s.v[k];
  s.q = lit<T>(0.5) * v2;
  s.e = (s.rhoE - s.rho * s.q) / s.rho;
  T p_rho, p_e;
  eos_p(M, s.rho, s.e, s.p, p_rho, p_e);
  s.c = sqrt_(p_rho + p_e * s.p / (s.rho * s.rho));
  s.H = (s.rhoE + s.p) / s.rho;
  for (int k = 0; k < 5; ++k) s.dp[k] = lit<T>(0.0);
  s.dp[0] = p_rho + p_e * (s.q - s.e) / s.rho;
  for (int k = 0; k < D; ++k) s.dp[1 + k] = -(p_e * s.v[k] / s.rho);
  s.dp[D + 1] = p_e / s.rho;
  return s;
}

// A_d = dF_d/dU under a general EOS, differentiating the flux of flux_d term
// by term with dp/dU from the state (u = v_d):
//   row 0    : e_{1+d}
//   row 1+i  : d(m_i u)/dU + delta_id dp/dU, with d(m_i u)/drho = -u v_i,
//              d(m_i u)/dm_j = delta_ij u + delta_jd v_i
//   row nv-1 : d(u rho H)/dU = u (dp/dU) + (-u H, delta_jd H, u)
template <class T> void jacobian_eos_d(const State<T>& s, int d, T* A) {
  const int D = s.D, nv = D + 2;
  const T zero = lit<T>(0.0), one = lit<T>(1.0);
  for (int k = 0; k < nv * nv; ++k) A[k] = zero;
  const T u = s.v[d];
  A[0 * nv + (1 + d)] = one;
  for (int i = 0; i < D; ++i) {
    T* row = A + (1 + i) * nv;
    row[0] = -(u * s.v[i]);
    for (int j = 0; j < D; ++j) {
      T e = zero;
      if (j == i) e = e + u;
      if (j == d) e = e + s.v[i];
      row[1 + j] = e;
    }
    if (i == d)
      for (int k = 0; k < nv; ++k) row[k] = row[k] + s.dp[k];
  }
  T* last = A + (nv - 1) * nv;
  last[0] = u * s.dp[0] - u * s.H;
  for (int j = 0; j < D; ++j) {
    last[1 + j] = u * s.dp[1 + j];
    if (j == d) last[1 + j] = last[1 + j] + s.H;
  }
  last[nv - 1] = u * s.dp[nv - 1] + u;
}

// Right eigenvectors of A_d under a general EOS (columns of R, eigenvalues
// u - c, u, ..., u, u + c):
//   r_1 = (1, v - c e_d, H - u c),  r_nv = (1, v + c e_d, H + u c),
//   r_2 = (1, v, eps) with eps fixed by dp/dU . r_2 = 0 (no pressure jump
//         across the entropy wave): eps = -(dp_rho + sum_j dp_mj v_j)/dp_rhoE,
//   r_{2+k} = (0, e_t, v_t)  (dp/dU . r = -p_e v_t/rho + p_e v_t/rho = 0).
template <class T> void right_eig_eos_d(const State<T>& s, int d, T* R, T* lam) {
  const int D = s.D, nv = D + 2;
  const T zero = lit<T>(0.0), one = lit<T>(1.0);
  const T u = s.v[d], c = s.c;
  for (int k = 0; k < nv * nv; ++k) R[k] = zero;
  R[0 * nv + 0] = one;
  for (int i = 0; i < D; ++i) R[(1 + i) * nv + 0] = (i == d) ? s.v[i] - c : s.v[i];
  R[(nv - 1) * nv + 0] = s.H - u * c;
  T num = s.dp[0];
  for (int j = 0; j < D; ++j) num = num + s.dp[1 + j] * s.v[j];
  R[0 * nv + 1] = one;
  for (int i = 0; i < D; ++i) R[(1 + i) * nv + 1] = s.v[i];
  R[(nv - 1) * nv + 1] = -(num / s.dp[nv - 1]);
  for (int k = 0; k < D - 1; ++k) {
    int t = tangential(D, d, k);
    R[(1 + t) * nv + (2 + k)] = one;
    R[(nv - 1) * nv + (2 + k)] = s.v[t];
  }
  R[0 * nv + (nv - 1)] = one;
  for (int i = 0; i < D; ++i) R[(1 + i) * nv + (nv - 1)] = (i == d) ? s.v[i] + c : s.v[i];
  R[(nv - 1) * nv + (nv - 1)] = s.H + u * c;
  if (lam) {
    lam[0] = u - c;
    for (int k = 1; k < nv - 1; ++k) lam[k] = u;
    lam[nv - 1] = u + c;
  }
}

// Left eigenvectors (rows of L = R^{-1}) under a general EOS, with
// beta = (dp/dU) / c^2 (a row vector):
//   l_1  = 1/2 (beta + (u/c) e_0 - (1/c) e_{1+d})
//   l_2  = e_0 - beta
//   l_{2+k} = -v_t e_0 + e_{1+t}
//   l_nv = 1/2 (beta - (u/c) e_0 + (1/c) e_{1+d})
// (the acoustic rows pick out (dp +- rho c du_d)/(2 c^2), the entropy row
// drho - dp/c^2).
template <class T> void left_eig_eos_d(const State<T>& s, int d, T* L) {
  const int D = s.D, nv = D + 2;
  const T zero = lit<T>(0.0), one = lit<T>(1.0), half = lit<T>(0.5);
  const T u = s.v[d], c = s.c;
  const T c2 = c * c;
  for (int k = 0; k < nv * nv; ++k) L[k] = zero;
  T* l1 = L + 0 * nv;
  T* l2 = L + 1 * nv;
  T* ln = L + (nv - 1) * nv;
  for (int k = 0; k < nv; ++k) {
    const T beta = s.dp[k] / c2;
    T a = beta, b = beta;
    if (k == 0) {
      a = a + u / c;
      b = b - u / c;
    } else if (k == 1 + d) {
      a = a - one / c;
      b = b + one / c;
    }
    l1[k] = half * a;
    ln[k] = half * b;
    l2[k] = (k == 0) ? one - beta : -beta;
  }
  for (int k = 0; k < D - 1; ++k) {
    int t = tangential(D, d, k);
    T* lk = L + (2 + k) * nv;
    lk[0] = -s.v[t];
    lk[1 + t] = one;
  }
}

// Flux from primitive variables under a general EOS:
//   F_d = (rho u, rho u v + p e_d, u (rho e(rho, p) + rho |v|^2 / 2 + p)).
template <class T>
void flux_prim_eos_d(int D, const EosModel& M, const double* const* V, int64_t i, int d, T* F) {
  const T rho = lit<T>(V[0][i]), p = lit<T>(V[D + 1][i]);
  T v[3];
  for (int k = 0; k < D; ++k) v[k] = lit<T>(V[1 + k][i]);
  T v2 = v[0] * v[0];
  for (int k = 1; k < D; ++k) v2 = v2 + v[k] * v[k];
  T z, z_rho, z_p;
  eos_rhoe(M, rho, p, z, z_rho, z_p);
  const T u = v[d];
  F[0] = rho * u;
  for (int k = 0; k < D; ++k) {
    F[1 + k] = rho * u * v[k];
    if (k == d) F[1 + k] = F[1 + k] + p;
  }
  F[D + 1] = u * (z + lit<T>(0.5) * rho * v2 + p);
}

// B_d = dF_d/dV under a general EOS (rows in U order, columns in V order):
// rows 0..D as for the ideal gas; row nv-1 differentiates
// u (z(rho, p) + rho |v|^2/2 + p):
//   (u (z_rho + |v|^2/2), delta_jd (z + rho |v|^2/2 + p) + rho u v_j, u (z_p + 1)).
template <class T>
void jac_prim_eos_d(int D, const EosModel& M, const double* const* V, int64_t i, int d, T* B) {
  const int nv = D + 2;
  const T zero = lit<T>(0.0), one = lit<T>(1.0);
  const T rho = lit<T>(V[0][i]), p = lit<T>(V[D + 1][i]);
  T v[3];
  for (int k = 0; k < D; ++k) v[k] = lit<T>(V[1 + k][i]);
  T v2 = v[0] * v[0];
  for (int k = 1; k < D; ++k) v2 = v2 + v[k] * v[k];
  T z, z_rho, z_p;
  eos_rhoe(M, rho, p, z, z_rho, z_p);
  const T u = v[d];
  for (int k = 0; k < nv * nv; ++k) B[k] = zero;
  B[0] = u;
  B[1 + d] = rho;
  for (int r = 0; r < D; ++r) {
    T* row = B + (1 + r) * nv;
    row[0] = u * v[r];
    for (int j = 0; j < D; ++j) {
      T e = zero;
      if (j == d) e = e + rho * v[r];
      if (j == r) e = e + rho * u;
      row[1 + j] = e;
    }
    row[nv - 1] = (r == d) ? one : zero;
  }
  T* last = B + (nv - 1) * nv;
  last[0] = u * (z_rho + lit<T>(0.5) * v2);
  for (int j = 0; j < D; ++j) {
    T e = rho * u * v[j];
    if (j == d) e = e + (z + lit<T>(0.5) * rho * v2 + p);
    last[1 + j] = e;
  }
  last[nv - 1] = u * (z_p + one);
}

// Array drivers of the general-EOS blocks (same layouts as the ideal-gas ones).
template <class T>
void run_eos_prim_from_cons(int D, const EosModel& M, int64_t n, const double* const* U, double* const* V,
                            double* const* sc) {
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    put(V, sc, 0, i, s.rho);
    for (int k = 0; k < D; ++k) put(V, sc, 1 + k, i, s.v[k]);
    put(V, sc, D + 1, i, s.p);
  }
}

template <class T>
void run_eos_cons_from_prim(int D, const EosModel& M, int64_t n, const double* const* V, double* const* U,
                            double* const* sc) {
  // m_i = rho v_i, rhoE = rho e(rho, p) + rho |v|^2 / 2.
  for (int64_t i = 0; i < n; ++i) {
    T rho = lit<T>(V[0][i]);
    T v2 = lit<T>(0.0);
    put(U, sc, 0, i, rho);
    for (int k = 0; k < D; ++k) {
      T vk = lit<T>(V[1 + k][i]);
      put(U, sc, 1 + k, i, rho * vk);
      v2 = (k == 0) ? vk * vk : v2 + vk * vk;
    }
    T z, z_rho, z_p;
    eos_rhoe(M, rho, lit<T>(V[D + 1][i]), z, z_rho, z_p);
    put(U, sc, D + 1, i, z + lit<T>(0.5) * rho * v2);
  }
}

template <class T>
void run_eos_pc(int D, const EosModel& M, int64_t n, const double* const* U, double* const* out,
                double* const* sc) {
  // out = {p, c}
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    put(out, sc, 0, i, s.p);
    put(out, sc, 1, i, s.c);
  }
}

template <class T>
void run_eos_temperature(int D, const EosModel& M, int64_t n, const double* const* U, double* const* out,
                         double* const* sc) {
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    put(out, sc, 0, i, eos_T(M, s.rho, s.e));
  }
}

template <class T>
void run_eos_flux(int D, int dir, const EosModel& M, int64_t n, const double* const* U, double* const* F,
                  double* const* sc) {
  const int nv = D + 2;
  T f[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    for (int d = 0; d < D; ++d) {
      if (dir >= 0 && d != dir) continue;
      flux_d(s, d, f);
      const int base = (dir < 0) ? d * nv : 0;
      for (int k = 0; k < nv; ++k) put(F, sc, base + k, i, f[k]);
    }
  }
}

template <class T>
void run_eos_flux_jac(int D, int d, const EosModel& M, int64_t n, const double* const* U, double* const* A,
                      double* const* sc) {
  const int nv = D + 2;
  T a[25];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    jacobian_eos_d(s, d, a);
    for (int k = 0; k < nv * nv; ++k) put(A, sc, k, i, a[k]);
  }
}

template <class T>
void run_eos_char(int D, int d, const EosModel& M, int inverse, int64_t n, const double* const* U,
                  const double* const* W, double* const* Y, double* const* sc) {
  const int nv = D + 2;
  T Mx[25], w[5], y[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    if (inverse)
      right_eig_eos_d(s, d, Mx, (T*)nullptr);
    else
      left_eig_eos_d(s, d, Mx);
    for (int k = 0; k < nv; ++k) w[k] = lit<T>(W[k][i]);
    matvec(nv, Mx, w, y);
    for (int k = 0; k < nv; ++k) put(Y, sc, k, i, y[k]);
  }
}

template <class T>
void run_eos_flux_vjp(int D, int d, const EosModel& M, int64_t n, const double* const* U,
                      const double* const* G, double* const* gU, double* const* sc) {
  const int nv = D + 2;
  T a[25], gg[5], y[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    jacobian_eos_d(s, d, a);
    for (int k = 0; k < nv; ++k) gg[k] = lit<T>(G[k][i]);
    matvec_t(nv, a, gg, y);
    for (int k = 0; k < nv; ++k) put(gU, sc, k, i, y[k]);
  }
}

template <class T>
void run_eos_fused(int D, int dj, const EosModel& M, int64_t n, const double* const* U, const double* const* W,
                   double* const* out, double* const* sc) {
  // run_eos_flux(dir=-1), run_eos_flux_jac and run_eos_char(forward) in turn.
  const int nv = D + 2;
  const int off_A = D * nv, off_Y = D * nv + nv * nv;
  T f[5], a[25], Mx[25], w[5], y[5];
  for (int64_t i = 0; i < n; ++i) {
    State<T> s = state_from_cons_eos<T>(D, M, U, i);
    for (int d = 0; d < D; ++d) {
      flux_d(s, d, f);
      for (int k = 0; k < nv; ++k) put(out, sc, d * nv + k, i, f[k]);
    }
    jacobian_eos_d(s, dj, a);
    for (int k = 0; k < nv * nv; ++k) put(out, sc, off_A + k, i, a[k]);
    left_eig_eos_d(s, dj, Mx);
    for (int k = 0; k < nv; ++k) w[k] = lit<T>(W[k][i]);
    matvec(nv, Mx, w, y);
    for (int k = 0; k < nv; ++k) put(out, sc, off_Y + k, i, y[k]);
  }
}

template <class T>
void run_eos_flux_prim(int D, int dir, const EosModel& M, int64_t n, const double* const* V, double* const* F,
                       double* const* sc) {
  const int nv = D + 2;
  T f[5];
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < D; ++d) {
      if (dir >= 0 && d != dir) continue;
      flux_prim_eos_d<T>(D, M, V, i, d, f);
      const int base = (dir < 0) ? d * nv : 0;
      for (int k = 0; k < nv; ++k) put(F, sc, base + k, i, f[k]);
    }
}

template <class T>
void run_eos_jac_prim(int D, int d, const EosModel& M, int64_t n, const double* const* V, double* const* B,
                      double* const* sc) {
  const int nv = D + 2;
  T b[25];
  for (int64_t i = 0; i < n; ++i) {
    jac_prim_eos_d<T>(D, M, V, i, d, b);
    for (int k = 0; k < nv * nv; ++k) put(B, sc, k, i, b[k]);
  }
}

// ---------------------------------------------------------------------------
// Explicit first-order finite-volume step with the Rusanov (local
// Lax-Friedrichs) numerical flux on a periodic n^3 grid over [0,1]^3.
// Cell (i,j,k) is point index (k*n + j)*n + i (x fastest).
//   face flux  Fh = (F_d(U_L) + F_d(U_R))/2 - s (U_R - U_L)/2,
//              s  = max(|u_L| + c_L, |u_R| + c_R), u = v_d;
//   update     U <- U - dt/dx sum_d (Fh_{d,+1/2} - Fh_{d,-1/2});
//   time step  dt = CFL dx / max_cells sum_d (|v_d| + c)
// (the inviscid flux is the paper's, section 2.2; the scheme is textbook,
// Toro section 8.3 and 10.5).
// ---------------------------------------------------------------------------

inline int64_t cell(int n, int i, int j, int k) {
  i = (i % n + n) % n;
  j = (j % n + n) % n;
  k = (k % n + n) % n;
  return ((int64_t)k * n + j) * n + i;
}

double rusanov_max_speed(int n, double g, const double* const* U) {
  const int64_t N = (int64_t)n * n * n;
  double smax = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    State<double> s = state_from_cons<double>(3, g, U, i);
    double sum = std::fabs(s.v[0]) + s.c;
    sum = sum + (std::fabs(s.v[1]) + s.c);
    sum = sum + (std::fabs(s.v[2]) + s.c);
    if (sum > smax) smax = sum;
  }
  return smax;
}

void rusanov_face_flux(double g, const double* const* U, int64_t iL, int64_t iR, int d,
                       double* Fh) {
  State<double> L = state_from_cons<double>(3, g, U, iL);
  State<double> R = state_from_cons<double>(3, g, U, iR);
  double fL[5], fR[5];
  flux_d(L, d, fL);
  flux_d(R, d, fR);
  double sL = std::fabs(L.v[d]) + L.c;
  double sR = std::fabs(R.v[d]) + R.c;
  double s = sL > sR ? sL : sR;
  for (int k = 0; k < 5; ++k) Fh[k] = 0.5 * (fL[k] + fR[k]) - 0.5 * s * (U[k][iR] - U[k][iL]);
}

void rusanov_step(int n, double g, double dt, const double* const* U, double* const* Unew) {
  const double dx = 1.0 / n;
  const double lam = dt / dx;
  double Fm[5], Fp[5];
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int64_t c = cell(n, i, j, k);
        double div[5] = {0, 0, 0, 0, 0};
        for (int d = 0; d < 3; ++d) {
          int64_t cm = (d == 0) ? cell(n, i - 1, j, k) : (d == 1) ? cell(n, i, j - 1, k) : cell(n, i, j, k - 1);
          int64_t cp = (d == 0) ? cell(n, i + 1, j, k) : (d == 1) ? cell(n, i, j + 1, k) : cell(n, i, j, k + 1);
          rusanov_face_flux(g, U, cm, c, d, Fm);
          rusanov_face_flux(g, U, c, cp, d, Fp);
          for (int q = 0; q < 5; ++q) div[q] = div[q] + (Fp[q] - Fm[q]);
        }
        for (int q = 0; q < 5; ++q) Unew[q][c] = U[q][c] - lam * div[q];
      }
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (loaded with ctypes by the tests).  Return 0 on success,
// 1 on a bad argument.  `scale` may be NULL; otherwise it holds one plane
// pointer per output plane and receives the running-error scale S.
// ---------------------------------------------------------------------------

extern "C" {

int oracle_v_mag2(int D, int64_t n, const double* const* U, double* const* out,
                  double* const* scale) {
  if (bad_dim(D) || n < 0) return 1;
  run_v_mag2<double>(D, n, U, out, nullptr);
  if (scale) run_v_mag2<Err>(D, n, U, nullptr, scale);
  return 0;
}

int oracle_prim_from_cons(int D, double g, int64_t n, const double* const* U, double* const* V,
                          double* const* scale) {
  if (bad_dim(D) || n < 0 || !(g > 1.0)) return 1;
  run_prim_from_cons<double>(D, g, n, U, V, nullptr);
  if (scale) run_prim_from_cons<Err>(D, g, n, U, nullptr, scale);
  return 0;
}

int oracle_cons_from_prim(int D, double g, int64_t n, const double* const* V, double* const* U,
                          double* const* scale) {
  if (bad_dim(D) || n < 0 || !(g > 1.0)) return 1;
  run_cons_from_prim<double>(D, g, n, V, U, nullptr);
  if (scale) run_cons_from_prim<Err>(D, g, n, V, nullptr, scale);
  return 0;
}

int oracle_eos(int D, double g, int64_t n, const double* const* U, double* const* out,
               double* const* scale) {
  if (bad_dim(D) || n < 0 || !(g > 1.0)) return 1;
  run_eos<double>(D, g, n, U, out, nullptr);
  if (scale) run_eos<Err>(D, g, n, U, nullptr, scale);
  return 0;
}

int oracle_riemann_inv(int D, int d, double g, int64_t n, const double* const* U,
                       double* const* out, double* const* scale) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  run_riemann<double>(D, d, g, n, U, out, nullptr);
  if (scale) run_riemann<Err>(D, d, g, n, U, nullptr, scale);
  return 0;
}

int oracle_flux(int D, int dir, double g, int64_t n, const double* const* U, double* const* F,
                double* const* scale) {
  if (bad_dim(D) || dir < -1 || dir >= D || n < 0 || !(g > 1.0)) return 1;
  run_flux<double>(D, dir, g, n, U, F, nullptr);
  if (scale) run_flux<Err>(D, dir, g, n, U, nullptr, scale);
  return 0;
}

int oracle_flux_jac(int D, int d, double g, int64_t n, const double* const* U, double* const* A,
                    double* const* scale) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  run_flux_jac<double>(D, d, g, n, U, A, nullptr);
  if (scale) run_flux_jac<Err>(D, d, g, n, U, nullptr, scale);
  return 0;
}

int oracle_char_transform(int D, int d, double g, int inverse, int64_t n, const double* const* U,
                          const double* const* W, double* const* Y, double* const* scale) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  run_char<double>(D, d, g, inverse, n, U, W, Y, nullptr);
  if (scale) run_char<Err>(D, d, g, inverse, n, U, W, nullptr, scale);
  return 0;
}

int oracle_flux_vjp(int D, int d, double g, int64_t n, const double* const* U,
                    const double* const* G, double* const* gU, double* const* scale) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  run_flux_vjp<double>(D, d, g, n, U, G, gU, nullptr);
  if (scale) run_flux_vjp<Err>(D, d, g, n, U, G, nullptr, scale);
  return 0;
}

int oracle_euler_fused(int D, int dj, double g, int64_t n, const double* const* U,
                       const double* const* W, double* const* out, double* const* scale) {
  if (bad_dim(D) || dj < 0 || dj >= D || n < 0 || !(g > 1.0)) return 1;
  run_fused<double>(D, dj, g, n, U, W, out, nullptr);
  if (scale) run_fused<Err>(D, dj, g, n, U, W, nullptr, scale);
  return 0;
}

int oracle_flux_prim(int D, int dir, double g, int64_t n, const double* const* V, double* const* F,
                     double* const* scale) {
  if (bad_dim(D) || dir < -1 || dir >= D || n < 0 || !(g > 1.0)) return 1;
  run_flux_prim<double>(D, dir, g, n, V, F, nullptr);
  if (scale) run_flux_prim<Err>(D, dir, g, n, V, nullptr, scale);
  return 0;
}

int oracle_flux_jac_prim(int D, int d, double g, int64_t n, const double* const* V, double* const* B,
                         double* const* scale) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  run_jac_prim<double>(D, d, g, n, V, B, nullptr);
  if (scale) run_jac_prim<Err>(D, d, g, n, V, nullptr, scale);
  return 0;
}

int oracle_temperature(int D, double g, double cv, int64_t n, const double* const* U, double* const* out,
                       double* const* scale) {
  if (bad_dim(D) || n < 0 || !(g > 1.0) || !(cv > 0.0)) return 1;
  run_temperature<double>(D, g, cv, n, U, out, nullptr);
  if (scale) run_temperature<Err>(D, g, cv, n, U, nullptr, scale);
  return 0;
}

int oracle_roe_flux(int D, int d, double g, int64_t n, const double* const* UL, const double* const* UR,
                    double* const* F, double* const* scale) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  run_roe_flux<double>(D, d, g, n, UL, UR, F, nullptr);
  if (scale) run_roe_flux<Err>(D, d, g, n, UL, UR, nullptr, scale);
  return 0;
}

int oracle_roe_char_transform(int D, int d, double g, int inverse, int64_t n, const double* const* UL,
                              const double* const* UR, const double* const* W, double* const* Y,
                              double* const* scale) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  run_roe_char<double>(D, d, g, inverse, n, UL, UR, W, Y, nullptr);
  if (scale) run_roe_char<Err>(D, d, g, inverse, n, UL, UR, W, nullptr, scale);
  return 0;
}

// Eigen-decomposition of A_d at each point: R (nv*nv planes, column k is the
// right eigenvector r_k), L = R^{-1} (nv*nv planes, row k is l_k), lambda (nv
// planes).  Any of R, L, lam may be NULL.
int oracle_eig(int D, int d, double g, int64_t n, const double* const* U, double* const* R,
               double* const* L, double* const* lam) {
  if (bad_dim(D) || d < 0 || d >= D || n < 0 || !(g > 1.0)) return 1;
  const int nv = D + 2;
  double r[25], l[25], lm[5];
  for (int64_t i = 0; i < n; ++i) {
    State<double> s = state_from_cons<double>(D, g, U, i);
    right_eig_d(s, d, r, lm);
    left_eig_d(s, d, l);
    for (int k = 0; k < nv * nv; ++k) {
      if (R && R[k]) R[k][i] = r[k];
      if (L && L[k]) L[k][i] = l[k];
    }
    for (int k = 0; k < nv; ++k)
      if (lam && lam[k]) lam[k][i] = lm[k];
  }
  return 0;
}

// General-EOS blocks.  `eos` = {kind (1 NASG, 2 van der Waals), gamma,
// p_inf, b, q, a, c_v}; outputs and layouts as for the ideal-gas blocks
// (eos_pc: {p, c}).
#define ORACLE_EOS_ARGS(cond)                      \
  EosModel M;                                      \
  if (bad_dim(D) || n < 0 || !eos_from_params(eos, M) || !(cond)) return 1;

int oracle_eos_prim_from_cons(const double* eos, int D, int64_t n, const double* const* U, double* const* V,
                              double* const* scale) {
  ORACLE_EOS_ARGS(true)
  run_eos_prim_from_cons<double>(D, M, n, U, V, nullptr);
  if (scale) run_eos_prim_from_cons<Err>(D, M, n, U, nullptr, scale);
  return 0;
}

int oracle_eos_cons_from_prim(const double* eos, int D, int64_t n, const double* const* V, double* const* U,
                              double* const* scale) {
  ORACLE_EOS_ARGS(true)
  run_eos_cons_from_prim<double>(D, M, n, V, U, nullptr);
  if (scale) run_eos_cons_from_prim<Err>(D, M, n, V, nullptr, scale);
  return 0;
}

int oracle_eos_pc(const double* eos, int D, int64_t n, const double* const* U, double* const* out,
                  double* const* scale) {
  ORACLE_EOS_ARGS(true)
  run_eos_pc<double>(D, M, n, U, out, nullptr);
  if (scale) run_eos_pc<Err>(D, M, n, U, nullptr, scale);
  return 0;
}

int oracle_eos_temperature(const double* eos, int D, int64_t n, const double* const* U, double* const* out,
                           double* const* scale) {
  ORACLE_EOS_ARGS(true)
  run_eos_temperature<double>(D, M, n, U, out, nullptr);
  if (scale) run_eos_temperature<Err>(D, M, n, U, nullptr, scale);
  return 0;
}

int oracle_eos_flux(const double* eos, int D, int dir, int64_t n, const double* const* U, double* const* F,
                    double* const* scale) {
  ORACLE_EOS_ARGS(dir >= -1 && dir < D)
  run_eos_flux<double>(D, dir, M, n, U, F, nullptr);
  if (scale) run_eos_flux<Err>(D, dir, M, n, U, nullptr, scale);
  return 0;
}

int oracle_eos_flux_jac(const double* eos, int D, int d, int64_t n, const double* const* U, double* const* A,
                        double* const* scale) {
  ORACLE_EOS_ARGS(d >= 0 && d < D)
  run_eos_flux_jac<double>(D, d, M, n, U, A, nullptr);
  if (scale) run_eos_flux_jac<Err>(D, d, M, n, U, nullptr, scale);
  return 0;
}

int oracle_eos_char_transform(const double* eos, int D, int d, int inverse, int64_t n, const double* const* U,
                              const double* const* W, double* const* Y, double* const* scale) {
  ORACLE_EOS_ARGS(d >= 0 && d < D)
  run_eos_char<double>(D, d, M, inverse, n, U, W, Y, nullptr);
  if (scale) run_eos_char<Err>(D, d, M, inverse, n, U, W, nullptr, scale);
  return 0;
}

int oracle_eos_flux_vjp(const double* eos, int D, int d, int64_t n, const double* const* U,
                        const double* const* G, double* const* gU, double* const* scale) {
  ORACLE_EOS_ARGS(d >= 0 && d < D)
  run_eos_flux_vjp<double>(D, d, M, n, U, G, gU, nullptr);
  if (scale) run_eos_flux_vjp<Err>(D, d, M, n, U, G, nullptr, scale);
  return 0;
}

int oracle_eos_euler_fused(const double* eos, int D, int dj, int64_t n, const double* const* U,
                           const double* const* W, double* const* out, double* const* scale) {
  ORACLE_EOS_ARGS(dj >= 0 && dj < D)
  run_eos_fused<double>(D, dj, M, n, U, W, out, nullptr);
  if (scale) run_eos_fused<Err>(D, dj, M, n, U, W, nullptr, scale);
  return 0;
}

int oracle_eos_flux_prim(const double* eos, int D, int dir, int64_t n, const double* const* V,
                         double* const* F, double* const* scale) {
  ORACLE_EOS_ARGS(dir >= -1 && dir < D)
  run_eos_flux_prim<double>(D, dir, M, n, V, F, nullptr);
  if (scale) run_eos_flux_prim<Err>(D, dir, M, n, V, nullptr, scale);
  return 0;
}

int oracle_eos_flux_jac_prim(const double* eos, int D, int d, int64_t n, const double* const* V,
                             double* const* B, double* const* scale) {
  ORACLE_EOS_ARGS(d >= 0 && d < D)
  run_eos_jac_prim<double>(D, d, M, n, V, B, nullptr);
  if (scale) run_eos_jac_prim<Err>(D, d, M, n, V, nullptr, scale);
  return 0;
}

// Eigen-decomposition under a general EOS (as oracle_eig), plus the raw EOS
// values at each point: aux = {p, p_rho, p_e, T, e} (any entry may be NULL).
int oracle_eos_eig(const double* eos, int D, int d, int64_t n, const double* const* U, double* const* R,
                   double* const* L, double* const* lam, double* const* aux) {
  ORACLE_EOS_ARGS(d >= 0 && d < D)
  const int nv = D + 2;
  double r[25], l[25], lm[5];
  for (int64_t i = 0; i < n; ++i) {
    State<double> s = state_from_cons_eos<double>(D, M, U, i);
    right_eig_eos_d(s, d, r, lm);
    left_eig_eos_d(s, d, l);
    for (int k = 0; k < nv * nv; ++k) {
      if (R && R[k]) R[k][i] = r[k];
      if (L && L[k]) L[k][i] = l[k];
    }
    for (int k = 0; k < nv; ++k)
      if (lam && lam[k]) lam[k][i] = lm[k];
    if (aux) {
      double p, p_rho, p_e;
      eos_p(M, s.rho, s.e, p, p_rho, p_e);
      const double vals[5] = {p, p_rho, p_e, eos_T(M, s.rho, s.e), s.e};
      for (int k = 0; k < 5; ++k)
        if (aux[k]) aux[k][i] = vals[k];
    }
  }
  return 0;
}

// The EOS functions at given (rho, e) or (rho, p) pairs:
//   out_pe = {p, p_rho, p_e, T} at (rho[i], e[i]);
//   out_z  = {rho e, d(rho e)/drho|_p, d(rho e)/dp|_rho} at (rho[i], p[i] = e[i]).
int oracle_eos_point(const double* eos, int64_t n, const double* rho, const double* e, double* const* out_pe,
                     double* const* out_z) {
  EosModel M;
  if (n < 0 || !eos_from_params(eos, M)) return 1;
  for (int64_t i = 0; i < n; ++i) {
    if (out_pe) {
      double p, p_rho, p_e;
      eos_p(M, rho[i], e[i], p, p_rho, p_e);
      const double v[4] = {p, p_rho, p_e, eos_T(M, rho[i], e[i])};
      for (int k = 0; k < 4; ++k)
        if (out_pe[k]) out_pe[k][i] = v[k];
    }
    if (out_z) {
      double z, z_rho, z_p;
      eos_rhoe(M, rho[i], e[i], z, z_rho, z_p);
      const double v[3] = {z, z_rho, z_p};
      for (int k = 0; k < 3; ++k)
        if (out_z[k]) out_z[k][i] = v[k];
    }
  }
  return 0;
}
#undef ORACLE_EOS_ARGS

// Rusanov finite-volume scheme on one periodic n^3 grid (FP64).
double oracle_rusanov_dt(int n, double g, double cfl, const double* const* U) {
  if (n < 1 || !(g > 1.0)) return -1.0;
  return cfl * (1.0 / n) / rusanov_max_speed(n, g, U);
}

int oracle_rusanov_step(int n, double g, double dt, const double* const* U, double* const* Unew) {
  if (n < 1 || !(g > 1.0)) return 1;
  rusanov_step(n, g, dt, U, Unew);
  return 0;
}

// `steps` steps, each with dt from the state at its start; U is updated in
// place (work holds 5 planes of n^3 doubles).  dts (may be NULL) receives
// the time step of every step.
int oracle_rusanov_run(int n, double g, double cfl, int steps, double* const* U, double* const* work,
                       double* dts) {
  if (n < 1 || steps < 0 || !(g > 1.0)) return 1;
  const int64_t N = (int64_t)n * n * n;
  for (int s = 0; s < steps; ++s) {
    double dt = cfl * (1.0 / n) / rusanov_max_speed(n, g, U);
    if (dts) dts[s] = dt;
    rusanov_step(n, g, dt, U, work);
    for (int q = 0; q < 5; ++q)
      for (int64_t i = 0; i < N; ++i) U[q][i] = work[q][i];
  }
  return 0;
}

}  // extern "C"
