"""FP64 CPU oracle for the FDBB Euler building blocks (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library (``paper_1809_09851_gb300``) never imports it, and it imports
nothing from the product library.

All fields are lists of 1-D float64 numpy arrays, one array per component
plane, in the paper's component order (section 2.2): conservative
U = (rho, m_1..m_D, rhoE), primitive V = (rho, v_1..v_D, p).

Every function returns ``out`` or, with ``scale=True``, ``(out, S)`` where S
holds, per output plane, the first-order running-error scale of the oracle's
formula (|computed - exact| <~ 2^-53 * S); parity tolerances are ``tol * S``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build as _build, library_path

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build()
        lib = ctypes.CDLL(path)
        i64, dbl, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        ci = ctypes.c_int
        sig = {
            "oracle_v_mag2": [ci, i64, vp, vp, vp],
            "oracle_prim_from_cons": [ci, dbl, i64, vp, vp, vp],
            "oracle_cons_from_prim": [ci, dbl, i64, vp, vp, vp],
            "oracle_eos": [ci, dbl, i64, vp, vp, vp],
            "oracle_riemann_inv": [ci, ci, dbl, i64, vp, vp, vp],
            "oracle_flux": [ci, ci, dbl, i64, vp, vp, vp],
            "oracle_flux_jac": [ci, ci, dbl, i64, vp, vp, vp],
            "oracle_char_transform": [ci, ci, dbl, ci, i64, vp, vp, vp, vp],
            "oracle_flux_vjp": [ci, ci, dbl, i64, vp, vp, vp, vp],
            "oracle_euler_fused": [ci, ci, dbl, i64, vp, vp, vp, vp],
            "oracle_eig": [ci, ci, dbl, i64, vp, vp, vp, vp],
            "oracle_roe_flux": [ci, ci, dbl, i64, vp, vp, vp, vp],
            "oracle_flux_prim": [ci, ci, dbl, i64, vp, vp, vp],
            "oracle_flux_jac_prim": [ci, ci, dbl, i64, vp, vp, vp],
            "oracle_temperature": [ci, dbl, dbl, i64, vp, vp, vp],
            "oracle_roe_char_transform": [ci, ci, dbl, ci, i64, vp, vp, vp, vp, vp],
            "oracle_rusanov_step": [ci, dbl, dbl, vp, vp],
            "oracle_rusanov_run": [ci, dbl, dbl, ci, vp, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ci
        eos_sig = {
            "oracle_eos_prim_from_cons": [vp, ci, i64, vp, vp, vp],
            "oracle_eos_cons_from_prim": [vp, ci, i64, vp, vp, vp],
            "oracle_eos_pc": [vp, ci, i64, vp, vp, vp],
            "oracle_eos_temperature": [vp, ci, i64, vp, vp, vp],
            "oracle_eos_flux": [vp, ci, ci, i64, vp, vp, vp],
            "oracle_eos_flux_jac": [vp, ci, ci, i64, vp, vp, vp],
            "oracle_eos_char_transform": [vp, ci, ci, ci, i64, vp, vp, vp, vp],
            "oracle_eos_flux_vjp": [vp, ci, ci, i64, vp, vp, vp, vp],
            "oracle_eos_euler_fused": [vp, ci, ci, i64, vp, vp, vp, vp],
            "oracle_eos_flux_prim": [vp, ci, ci, i64, vp, vp, vp],
            "oracle_eos_flux_jac_prim": [vp, ci, ci, i64, vp, vp, vp],
            "oracle_eos_eig": [vp, ci, ci, i64, vp, vp, vp, vp, vp],
            "oracle_eos_point": [vp, i64, vp, vp, vp, vp],
        }
        for name, args in eos_sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ci
        lib.oracle_rusanov_dt.argtypes = [ci, dbl, dbl, vp]
        lib.oracle_rusanov_dt.restype = dbl
        _lib = lib
    return _lib


def _planes(arrs, n=None):
    """Validate a list of planes and return (ctypes pointer array, arrays, n)."""
    out = []
    for a in arrs:
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.ndim != 1:
            raise ValueError("planes must be 1-D")
        if n is None:
            n = a.shape[0]
        elif a.shape[0] != n:
            raise ValueError("planes differ in length")
        out.append(a)
    ptrs = (ctypes.c_void_p * len(out))(*[a.ctypes.data for a in out])
    return ptrs, out, n


def _new(k, n):
    arrs = [np.empty(n, dtype=np.float64) for _ in range(k)]
    ptrs = (ctypes.c_void_p * k)(*[a.ctypes.data for a in arrs])
    return ptrs, arrs


def _call(fn, nout, n, args, scale):
    po, out = _new(nout, n)
    ps, sc = _new(nout, n) if scale else (None, None)
    rc = fn(*args, po, ps)
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments ({fn.__name__})")
    return (out, sc) if scale else out


def nv(D: int) -> int:
    return D + 2


def v_mag2(D, U, scale=False):
    """|v|^2 = sum m_i^2 / rho^2 (paper section 3, Eq. (2))."""
    pu, Uk, n = _planes(U[: D + 1])
    return _call(_load().oracle_v_mag2, 1, n, (D, n, pu), scale)


def prim_from_cons(D, gamma, U, scale=False):
    pu, Uk, n = _planes(U)
    return _call(_load().oracle_prim_from_cons, nv(D), n, (D, gamma, n, pu), scale)


def cons_from_prim(D, gamma, V, scale=False):
    pv, Vk, n = _planes(V)
    return _call(_load().oracle_cons_from_prim, nv(D), n, (D, gamma, n, pv), scale)


def eos(D, gamma, U, scale=False):
    """[p, c]."""
    pu, Uk, n = _planes(U)
    return _call(_load().oracle_eos, 2, n, (D, gamma, n, pu), scale)


def riemann_inv(D, d, gamma, U, scale=False):
    """[w-, w+, s] along direction d."""
    pu, Uk, n = _planes(U)
    return _call(_load().oracle_riemann_inv, 3, n, (D, d, gamma, n, pu), scale)


def flux(D, d, gamma, U, scale=False):
    """F_d (nv planes) or, for d == -1, all directions (D*nv planes)."""
    pu, Uk, n = _planes(U)
    k = nv(D) * (D if d < 0 else 1)
    return _call(_load().oracle_flux, k, n, (D, d, gamma, n, pu), scale)


def flux_jac(D, d, gamma, U, scale=False):
    """A_d row-major, nv*nv planes."""
    pu, Uk, n = _planes(U)
    return _call(_load().oracle_flux_jac, nv(D) ** 2, n, (D, d, gamma, n, pu), scale)


def char_transform(D, d, gamma, U, W, inverse=False, scale=False):
    """Forward L_d(U) W or inverse R_d(U) W."""
    pu, Uk, n = _planes(U)
    pw, Wk, _ = _planes(W, n)
    return _call(_load().oracle_char_transform, nv(D), n,
                 (D, d, gamma, int(bool(inverse)), n, pu, pw), scale)


def flux_vjp(D, d, gamma, U, G, scale=False):
    """A_d(U)^T G."""
    pu, Uk, n = _planes(U)
    pg, Gk, _ = _planes(G, n)
    return _call(_load().oracle_flux_vjp, nv(D), n, (D, d, gamma, n, pu, pg), scale)


def euler_fused(D, dj, gamma, U, W, scale=False):
    """[F_0..F_{D-1} (D*nv), A_dj (nv*nv), L_dj W (nv)]."""
    pu, Uk, n = _planes(U)
    pw, Wk, _ = _planes(W, n)
    k = D * nv(D) + nv(D) ** 2 + nv(D)
    return _call(_load().oracle_euler_fused, k, n, (D, dj, gamma, n, pu, pw), scale)


def flux_prim(D, d, gamma, V, scale=False):
    """Inviscid flux from primitive variables V (F_d, or all directions for d == -1)."""
    pv, Vk, n = _planes(V)
    k = nv(D) * (D if d < 0 else 1)
    return _call(_load().oracle_flux_prim, k, n, (D, d, gamma, n, pv), scale)


def flux_jac_prim(D, d, gamma, V, scale=False):
    """dF_d/dV, nv*nv planes row-major (rows in U order, columns in V order)."""
    pv, Vk, n = _planes(V)
    return _call(_load().oracle_flux_jac_prim, nv(D) ** 2, n, (D, d, gamma, n, pv), scale)


def temperature(D, gamma, cv, U, scale=False):
    """[T] with T = e / c_v."""
    pu, Uk, n = _planes(U)
    return _call(_load().oracle_temperature, 1, n, (D, gamma, cv, n, pu), scale)


def roe_flux(D, d, gamma, UL, UR, scale=False):
    """Roe flux between UL and UR in direction d (nv planes)."""
    pl, Lk, n = _planes(UL)
    pr, Rk, _ = _planes(UR, n)
    return _call(_load().oracle_roe_flux, nv(D), n, (D, d, gamma, n, pl, pr), scale)


def roe_char_transform(D, d, gamma, UL, UR, W, inverse=False, scale=False):
    """L^ W (or R^ W) at the Roe-averaged state of (UL, UR)."""
    pl, Lk, n = _planes(UL)
    pr, Rk, _ = _planes(UR, n)
    pw, Wk, _ = _planes(W, n)
    return _call(_load().oracle_roe_char_transform, nv(D), n,
                 (D, d, gamma, int(bool(inverse)), n, pl, pr, pw), scale)


def eig(D, d, gamma, U):
    """(R, L, lam): R columns are right eigenvectors, L = R^-1, as plane lists."""
    pu, Uk, n = _planes(U)
    k = nv(D)
    pr, R = _new(k * k, n)
    pl, L = _new(k * k, n)
    pm, lam = _new(k, n)
    if _load().oracle_eig(D, d, gamma, n, pu, pr, pl, pm) != 0:
        raise ValueError("oracle rejected the arguments (oracle_eig)")
    return R, L, lam


def rusanov_dt(n, gamma, cfl, U):
    pu, Uk, N = _planes(U)
    assert N == n ** 3
    return _load().oracle_rusanov_dt(n, gamma, cfl, pu)


def rusanov_step(n, gamma, dt, U):
    pu, Uk, N = _planes(U)
    assert N == n ** 3
    po, out = _new(5, N)
    if _load().oracle_rusanov_step(n, gamma, dt, pu, po) != 0:
        raise ValueError("oracle rejected the arguments (oracle_rusanov_step)")
    return out


def rusanov_run(n, gamma, cfl, steps, U):
    """Run `steps` Rusanov steps; returns (U_final, dts)."""
    _, Uk, N = _planes(U)
    Uk = [a.copy() for a in Uk]
    pu = (ctypes.c_void_p * 5)(*[a.ctypes.data for a in Uk])
    pw, work = _new(5, N)
    dts = np.empty(max(steps, 1), dtype=np.float64)
    rc = _load().oracle_rusanov_run(n, gamma, cfl, steps, pu, pw,
                                    ctypes.c_void_p(dts.ctypes.data))
    if rc != 0:
        raise ValueError("oracle rejected the arguments (oracle_rusanov_run)")
    return Uk, dts[:steps]


# ---------------------------------------------------------------------------
# General equations of state (paper section 2.2, "Equations of state").
# An EOS is a dict: {"kind": "nasg", "gamma", "p_inf", "b", "q", "cv"} (the
# Noble-Abel stiffened gas) or {"kind": "vdw", "gamma", "a", "b", "cv"} (van
# der Waals); missing parameters are 0 (cv: 1).
# ---------------------------------------------------------------------------

_EOS_KINDS = {"nasg": 1, "vdw": 2}


def _eos(eos):
    kind = _EOS_KINDS[eos["kind"]]
    prm = np.array([kind, eos["gamma"], eos.get("p_inf", 0.0), eos.get("b", 0.0), eos.get("q", 0.0),
                    eos.get("a", 0.0), eos.get("cv", 1.0)], dtype=np.float64)
    return prm, ctypes.c_void_p(prm.ctypes.data)


def _call_eos(name, eos, nout, n, args, scale):
    prm, pp = _eos(eos)
    po, out = _new(nout, n)
    ps, sc = _new(nout, n) if scale else (None, None)
    rc = getattr(_load(), name)(pp, *args, po, ps)
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments ({name})")
    return (out, sc) if scale else out


def eos_prim_from_cons(eos, D, U, scale=False):
    pu, Uk, n = _planes(U)
    return _call_eos("oracle_eos_prim_from_cons", eos, nv(D), n, (D, n, pu), scale)


def eos_cons_from_prim(eos, D, V, scale=False):
    pv, Vk, n = _planes(V)
    return _call_eos("oracle_eos_cons_from_prim", eos, nv(D), n, (D, n, pv), scale)


def eos_pc(eos, D, U, scale=False):
    """[p, c] under a general EOS."""
    pu, Uk, n = _planes(U)
    return _call_eos("oracle_eos_pc", eos, 2, n, (D, n, pu), scale)


def eos_temperature(eos, D, U, scale=False):
    pu, Uk, n = _planes(U)
    return _call_eos("oracle_eos_temperature", eos, 1, n, (D, n, pu), scale)


def eos_flux(eos, D, d, U, scale=False):
    pu, Uk, n = _planes(U)
    k = nv(D) * (D if d < 0 else 1)
    return _call_eos("oracle_eos_flux", eos, k, n, (D, d, n, pu), scale)


def eos_flux_jac(eos, D, d, U, scale=False):
    pu, Uk, n = _planes(U)
    return _call_eos("oracle_eos_flux_jac", eos, nv(D) ** 2, n, (D, d, n, pu), scale)


def eos_char_transform(eos, D, d, U, W, inverse=False, scale=False):
    pu, Uk, n = _planes(U)
    pw, Wk, _ = _planes(W, n)
    return _call_eos("oracle_eos_char_transform", eos, nv(D), n, (D, d, int(bool(inverse)), n, pu, pw), scale)


def eos_flux_vjp(eos, D, d, U, G, scale=False):
    pu, Uk, n = _planes(U)
    pg, Gk, _ = _planes(G, n)
    return _call_eos("oracle_eos_flux_vjp", eos, nv(D), n, (D, d, n, pu, pg), scale)


def eos_euler_fused(eos, D, dj, U, W, scale=False):
    pu, Uk, n = _planes(U)
    pw, Wk, _ = _planes(W, n)
    k = D * nv(D) + nv(D) ** 2 + nv(D)
    return _call_eos("oracle_eos_euler_fused", eos, k, n, (D, dj, n, pu, pw), scale)


def eos_flux_prim(eos, D, d, V, scale=False):
    pv, Vk, n = _planes(V)
    k = nv(D) * (D if d < 0 else 1)
    return _call_eos("oracle_eos_flux_prim", eos, k, n, (D, d, n, pv), scale)


def eos_flux_jac_prim(eos, D, d, V, scale=False):
    pv, Vk, n = _planes(V)
    return _call_eos("oracle_eos_flux_jac_prim", eos, nv(D) ** 2, n, (D, d, n, pv), scale)


def eos_eig(eos, D, d, U):
    """(R, L, lam, aux) with aux = [p, p_rho, p_e, T, e] per point."""
    prm, pp = _eos(eos)
    pu, Uk, n = _planes(U)
    k = nv(D)
    pr, R = _new(k * k, n)
    pl, L = _new(k * k, n)
    pm, lam = _new(k, n)
    pa, aux = _new(5, n)
    if _load().oracle_eos_eig(pp, D, d, n, pu, pr, pl, pm, pa) != 0:
        raise ValueError("oracle rejected the arguments (oracle_eos_eig)")
    return R, L, lam, aux


def eos_point(eos, rho, e):
    """EOS functions at points: ([p, p_rho, p_e, T] at (rho, e),
    [rho e, d(rho e)/drho|_p, d(rho e)/dp|_rho] at (rho, p = e))."""
    prm, pp = _eos(eos)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    n = rho.shape[0]
    p1, a = _new(4, n)
    p2, z = _new(3, n)
    if _load().oracle_eos_point(pp, n, ctypes.c_void_p(rho.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                                p1, p2) != 0:
        raise ValueError("oracle rejected the arguments (oracle_eos_point)")
    return a, z


__all__ = [
    "v_mag2", "prim_from_cons", "cons_from_prim", "eos", "riemann_inv", "flux",
    "flux_jac", "char_transform", "flux_vjp", "euler_fused", "eig", "rusanov_dt",
    "rusanov_step", "rusanov_run", "roe_flux", "roe_char_transform", "flux_prim", "flux_jac_prim", "temperature",
    "eos_prim_from_cons", "eos_cons_from_prim", "eos_pc", "eos_temperature", "eos_flux", "eos_flux_jac",
    "eos_char_transform", "eos_flux_vjp", "eos_euler_fused", "eos_flux_prim", "eos_flux_jac_prim", "eos_eig",
    "eos_point", "library_path", "nv",
]
