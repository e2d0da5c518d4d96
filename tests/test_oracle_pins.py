"""Pins of the FP64 CPU oracle against facts it does not compute itself.

Every oracle function is checked against at least one of: hand-derived values
(tests/golden/euler_hand_values.txt), an identity of the Euler algebra
(round trips, homogeneity A(U) U = F(U), L R = I, A r = lambda r), a library
routine (numpy matrix inverse / matmul), central finite differences, or a
symmetry (axis permutation).  Each is chosen so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one test.
"""
import ast
import math
import operator
import os

import numpy as np
import pytest

import oracle
from paper_1809_09851_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "euler_hand_values.txt")
GAMMA = 1.4


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

_OPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul,
        ast.Div: operator.truediv, ast.USub: operator.neg, ast.UAdd: operator.pos}


def _eval(expr: str) -> float:
    """Evaluate a golden expression: numbers, + - * /, parentheses, sqrt()."""
    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant):
            return float(node.value)
        if isinstance(node, ast.BinOp):
            return _OPS[type(node.op)](ev(node.left), ev(node.right))
        if isinstance(node, ast.UnaryOp):
            return _OPS[type(node.op)](ev(node.operand))
        if isinstance(node, ast.Call) and node.func.id == "sqrt":
            return math.sqrt(ev(node.args[0]))
        raise ValueError(expr)
    return ev(ast.parse(expr, mode="eval"))


def _golden():
    cases, values = {}, []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                name, D, g = tok[1], int(tok[2]), float(tok[3])
                cases[name] = (D, g, [float(x) for x in tok[4:]])
            else:
                values.append((tok[0], tok[1], int(tok[2]), _eval(tok[3])))
    return cases, values


def _state(V, D, g):
    U = oracle.cons_from_prim(D, g, [np.array([x]) for x in V])
    return U


def _quantity(case, qty, D, g, U):
    nv = D + 2
    if qty == "U":
        return [u[0] for u in U]
    if qty == "V":
        return [v[0] for v in oracle.prim_from_cons(D, g, U)]
    if qty == "p":
        return [oracle.eos(D, g, U)[0][0]]
    if qty == "c":
        return [oracle.eos(D, g, U)[1][0]]
    if qty == "H":
        # H = (rhoE + p)/rho is not an output of its own; it is the last
        # entry of the entropy eigenvector's partner: R[nv-1, 0] + u c
        R, L, lam = oracle.eig(D, 0, g, U)
        c = oracle.eos(D, g, U)[1][0]
        u = oracle.prim_from_cons(D, g, U)[1][0]
        return [R[(nv - 1) * nv + 0][0] + u * c]
    if qty == "vmag2":
        return [oracle.v_mag2(D, U)[0][0]]
    if qty == "s":
        return [oracle.riemann_inv(D, 0, g, U)[2][0]]
    d = int(qty[-1])
    q = qty[:-1]
    if q == "F":
        return [f[0] for f in oracle.flux(D, d, g, U)]
    if q == "A":
        return [a[0] for a in oracle.flux_jac(D, d, g, U)]
    if q == "wm":
        return [oracle.riemann_inv(D, d, g, U)[0][0]]
    if q == "wp":
        return [oracle.riemann_inv(D, d, g, U)[1][0]]
    R, L, lam = oracle.eig(D, d, g, U)
    if q == "R":
        return [r[0] for r in R]
    if q == "L":
        return [x[0] for x in L]
    if q == "lam":
        return [x[0] for x in lam]
    raise KeyError(qty)


def _rand_U(n, D, seed=7):
    V = synth.euler3d(n, seed=seed, D=D) if D > 1 else synth.euler1d(n, seed=seed)
    return oracle.cons_from_prim(D, GAMMA, V), V


def _perm_matrix(D, a, b):
    """Permutation of the state vector that swaps velocity components a and b."""
    nv = D + 2
    P = np.eye(nv)
    P[[1 + a, 1 + b]] = P[[1 + b, 1 + a]]
    return P


def _stack(planes):
    return np.stack(planes, axis=-1)  # (n, k)


# ---------------------------------------------------------------------------
# hand-derived values
# ---------------------------------------------------------------------------

def test_golden_values():
    cases, values = _golden()
    assert len(values) > 100
    states = {name: (D, g, _state(V, D, g)) for name, (D, g, V) in cases.items()}
    cache = {}
    for case, qty, idx, expect in values:
        D, g, U = states[case]
        key = (case, qty)
        if key not in cache:
            cache[key] = _quantity(case, qty, D, g, U)
        got = cache[key][idx]
        assert got == pytest.approx(expect, rel=1e-14, abs=1e-14), (case, qty, idx)


# ---------------------------------------------------------------------------
# variables and EOS
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_cons_prim_round_trip(D):
    U, V = _rand_U(4096, D)
    V2 = oracle.prim_from_cons(D, GAMMA, U)
    U2 = oracle.cons_from_prim(D, GAMMA, V2)
    for k in range(D + 2):
        np.testing.assert_allclose(V2[k], V[k], rtol=5e-13, atol=1e-13)
        np.testing.assert_allclose(U2[k], U[k], rtol=5e-13, atol=1e-13)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_eos_consistent_with_primitives(D):
    U, V = _rand_U(2048, D)
    p, c = oracle.eos(D, GAMMA, U)
    np.testing.assert_allclose(p, V[D + 1], rtol=5e-13)
    # c^2 rho / gamma = p for the perfect gas
    np.testing.assert_allclose(c * c * V[0] / GAMMA, V[D + 1], rtol=1e-13)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_v_mag2_matches_velocity(D):
    U, V = _rand_U(2048, D)
    y = oracle.v_mag2(D, U)[0]
    ref = sum(V[1 + k] ** 2 for k in range(D))
    np.testing.assert_allclose(y, ref, rtol=1e-13)


# ---------------------------------------------------------------------------
# fluxes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_flux_rest_state(D):
    n = 64
    V = synth.euler3d(n, seed=3, D=D)
    for k in range(D):
        V[1 + k][:] = 0.0
    U = oracle.cons_from_prim(D, GAMMA, V)
    p = oracle.eos(D, GAMMA, U)[0]
    np.testing.assert_allclose(p, V[D + 1], rtol=1e-15)
    for d in range(D):
        F = oracle.flux(D, d, GAMMA, U)
        for k in range(D + 2):
            expect = p if k == 1 + d else np.zeros(n)
            np.testing.assert_array_equal(F[k], expect)


@pytest.mark.parametrize("D", [2, 3])
def test_flux_and_jacobian_axis_permutation(D):
    """F_b(U) = P F_a(P U) and A_b(U) = P A_a(P U) P for the swap P of a, b."""
    U, _ = _rand_U(512, D)
    nv = D + 2
    for a in range(D):
        for b in range(D):
            if a == b:
                continue
            P = _perm_matrix(D, a, b)
            PU = [(_stack(U) @ P.T)[:, k] for k in range(nv)]
            Fa = _stack(oracle.flux(D, a, GAMMA, PU))
            Fb = _stack(oracle.flux(D, b, GAMMA, U))
            np.testing.assert_allclose(Fa @ P.T, Fb, rtol=1e-13, atol=1e-12)
            Aa = _stack(oracle.flux_jac(D, a, GAMMA, PU)).reshape(-1, nv, nv)
            Ab = _stack(oracle.flux_jac(D, b, GAMMA, U)).reshape(-1, nv, nv)
            np.testing.assert_allclose(P @ Aa @ P, Ab, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_flux_all_directions_layout(D):
    U, _ = _rand_U(300, D)
    nv = D + 2
    Fall = oracle.flux(D, -1, GAMMA, U)
    assert len(Fall) == D * nv
    for d in range(D):
        Fd = oracle.flux(D, d, GAMMA, U)
        for k in range(nv):
            np.testing.assert_array_equal(Fall[d * nv + k], Fd[k])


# ---------------------------------------------------------------------------
# Jacobians
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_jacobian_homogeneity(D):
    """Euler's theorem: F is homogeneous of degree 1 in U, so A(U) U = F(U)."""
    U, _ = _rand_U(2048, D)
    nv = D + 2
    Us = _stack(U)
    for d in range(D):
        A = _stack(oracle.flux_jac(D, d, GAMMA, U)).reshape(-1, nv, nv)
        F = _stack(oracle.flux(D, d, GAMMA, U))
        AU = np.einsum("nij,nj->ni", A, Us)
        scale = np.einsum("nij,nj->ni", np.abs(A), np.abs(Us))
        assert np.all(np.abs(AU - F) <= 1e-13 * scale)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_jacobian_central_differences(D):
    U, _ = _rand_U(256, D, seed=11)
    nv = D + 2
    for d in range(D):
        A = _stack(oracle.flux_jac(D, d, GAMMA, U)).reshape(-1, nv, nv)
        for j in range(nv):
            h = 1e-6 * np.maximum(1.0, np.abs(U[j]))
            Up = [u.copy() for u in U]
            Um = [u.copy() for u in U]
            Up[j] += h
            Um[j] -= h
            Fp = _stack(oracle.flux(D, d, GAMMA, Up))
            Fm = _stack(oracle.flux(D, d, GAMMA, Um))
            fd = (Fp - Fm) / (2 * h)[:, None]
            scale = np.abs(A).max(axis=(1, 2))[:, None] + 1.0
            assert np.all(np.abs(fd - A[:, :, j]) <= 1e-6 * scale), (d, j)


# ---------------------------------------------------------------------------
# eigen-structure and characteristic transform
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_eigenvectors(D):
    U, _ = _rand_U(1024, D, seed=5)
    nv = D + 2
    I = np.eye(nv)
    for d in range(D):
        R, L, lam = oracle.eig(D, d, GAMMA, U)
        R = _stack(R).reshape(-1, nv, nv)
        L = _stack(L).reshape(-1, nv, nv)
        lam = _stack(lam)
        A = _stack(oracle.flux_jac(D, d, GAMMA, U)).reshape(-1, nv, nv)
        # L R = I
        np.testing.assert_allclose(L @ R, np.broadcast_to(I, L.shape), atol=1e-12)
        # closed-form L equals the numerical inverse of R (numpy LU)
        Linv = np.linalg.inv(R)
        np.testing.assert_allclose(L, Linv, rtol=1e-10, atol=1e-10)
        # A r_k = lambda_k r_k
        AR = A @ R
        scale = np.abs(A) @ np.abs(R) + 1.0
        assert np.all(np.abs(AR - R * lam[:, None, :]) <= 1e-12 * scale)
        # R Lambda L = A
        RLL = (R * lam[:, None, :]) @ L
        assert np.all(np.abs(RLL - A) <= 1e-11 * (np.abs(A) + 1.0))
        # eigenvalues are u - c, u, ..., u + c
        Vp = oracle.prim_from_cons(D, GAMMA, U)
        c = oracle.eos(D, GAMMA, U)[1]
        np.testing.assert_allclose(lam[:, 0], Vp[1 + d] - c, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(lam[:, -1], Vp[1 + d] + c, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_char_transform(D):
    U, _ = _rand_U(512, D, seed=9)
    nv = D + 2
    n = U[0].shape[0]
    W = synth.char_weights(n, nv)
    for d in range(D):
        R, L, lam = oracle.eig(D, d, GAMMA, U)
        Rm = _stack(R).reshape(-1, nv, nv)
        # forward on a right eigenvector gives the unit vector
        for k in range(nv):
            rk = [Rm[:, i, k] for i in range(nv)]
            Y = _stack(oracle.char_transform(D, d, GAMMA, U, rk))
            np.testing.assert_allclose(Y, np.broadcast_to(np.eye(nv)[k], Y.shape), atol=1e-11)
        # inverse reproduces R W (numpy matmul) and undoes forward
        Yinv = _stack(oracle.char_transform(D, d, GAMMA, U, W, inverse=True))
        np.testing.assert_allclose(Yinv, np.einsum("nij,nj->ni", Rm, _stack(W)), rtol=1e-12, atol=1e-12)
        Yf = oracle.char_transform(D, d, GAMMA, U, W)
        back = _stack(oracle.char_transform(D, d, GAMMA, U, Yf, inverse=True))
        np.testing.assert_allclose(back, _stack(W), rtol=1e-10, atol=1e-10)


# ---------------------------------------------------------------------------
# Riemann invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_riemann_invariants(D):
    U, V = _rand_U(2048, D, seed=13)
    c = oracle.eos(D, GAMMA, U)[1]
    for d in range(D):
        wm, wp, s = oracle.riemann_inv(D, d, GAMMA, U)
        np.testing.assert_allclose(wp - wm, 4 * c / (GAMMA - 1), rtol=1e-13)
        np.testing.assert_allclose(0.5 * (wp + wm), V[1 + d], rtol=1e-12, atol=1e-12)
        # entropy is invariant under rho -> k rho, p -> k^gamma p
        k = 1.7
        V2 = [V[0] * k, *V[1:D + 1], V[D + 1] * k ** GAMMA]
        s2 = oracle.riemann_inv(D, d, GAMMA, oracle.cons_from_prim(D, GAMMA, V2))[2]
        np.testing.assert_allclose(s2, s, rtol=1e-12)


# ---------------------------------------------------------------------------
# VJP and fused
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_flux_vjp(D):
    U, _ = _rand_U(256, D, seed=17)
    nv = D + 2
    n = U[0].shape[0]
    G = synth.cotangent(n, nv)
    for d in range(D):
        gU = _stack(oracle.flux_vjp(D, d, GAMMA, U, G))
        A = _stack(oracle.flux_jac(D, d, GAMMA, U)).reshape(-1, nv, nv)
        np.testing.assert_allclose(gU, np.einsum("nij,ni->nj", A, _stack(G)), rtol=1e-12, atol=1e-12)
        # central differences of <G, F_d(U)>
        for j in range(nv):
            h = 1e-6 * np.maximum(1.0, np.abs(U[j]))
            Up = [u.copy() for u in U]
            Um = [u.copy() for u in U]
            Up[j] += h
            Um[j] -= h
            fp = (_stack(oracle.flux(D, d, GAMMA, Up)) * _stack(G)).sum(axis=1)
            fm = (_stack(oracle.flux(D, d, GAMMA, Um)) * _stack(G)).sum(axis=1)
            fd = (fp - fm) / (2 * h)
            scale = (np.abs(A).sum(axis=1) * np.abs(_stack(G))).sum(axis=1) + 1.0
            assert np.all(np.abs(fd - gU[:, j]) <= 1e-6 * scale)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_fused_is_the_composition(D):
    U, _ = _rand_U(300, D, seed=19)
    nv = D + 2
    W = synth.char_weights(U[0].shape[0], nv)
    for dj in range(D):
        out = oracle.euler_fused(D, dj, GAMMA, U, W)
        ref = (oracle.flux(D, -1, GAMMA, U) + oracle.flux_jac(D, dj, GAMMA, U)
               + oracle.char_transform(D, dj, GAMMA, U, W))
        assert len(out) == len(ref) == D * nv + nv * nv + nv
        for a, b in zip(out, ref):
            np.testing.assert_array_equal(a, b)


def test_error_scale_bounds_value_and_flags_cancellation():
    """S >= |o| everywhere, and S >> |p| where rhoE - rho q cancels."""
    V = synth.euler3d(256, seed=23)
    V[1][:128] = 300.0  # high speed: rho q >> rho e
    U = oracle.cons_from_prim(3, GAMMA, V)
    out, S = oracle.euler_fused(3, 0, GAMMA, U, synth.char_weights(256), scale=True)
    for o, s in zip(out, S):
        # S == 0 only where the output is an exact copy of an input (F_d[0] = m_d)
        assert np.all((s >= np.abs(o) * (1 - 1e-15)) | (s == 0))
    assert np.all(S[0] == 0) and np.all(S[1] > 0)
    (p, c), (Sp, Sc) = oracle.eos(3, GAMMA, U, scale=True)
    assert np.all(Sp[:128] > 100 * np.abs(p[:128]))
    assert np.all(Sp[128:] < 1e4 * np.abs(p[128:]))


def test_argument_checks():
    U, _ = _rand_U(8, 3)
    with pytest.raises(ValueError):
        oracle.flux(3, 3, GAMMA, U)
    with pytest.raises(ValueError):
        oracle.flux_jac(3, 0, 1.0, U)


# ---------------------------------------------------------------------------
# Rusanov finite-volume step
# ---------------------------------------------------------------------------

def _fv_init(n, seed=31, vel=0.0):
    V = synth.smooth_perturbation(n, seed)
    V[1] = V[1] + vel
    return oracle.cons_from_prim(3, GAMMA, V)


def test_rusanov_conservation_and_uniform_state():
    n = 8
    U = _fv_init(n)
    U2, dts = oracle.rusanov_run(n, GAMMA, 0.4, 5, U)
    for k in range(5):
        assert abs(U2[k].sum() - U[k].sum()) <= 1e-12 * max(1.0, np.abs(U[k]).sum())
    assert np.all(dts > 0)
    # uniform state with velocity is preserved exactly
    V = [np.full(n ** 3, 1.3), np.full(n ** 3, 0.4), np.full(n ** 3, -0.2), np.full(n ** 3, 0.1),
         np.full(n ** 3, 0.9)]
    Uu = oracle.cons_from_prim(3, GAMMA, V)
    Uu2, dts = oracle.rusanov_run(n, GAMMA, 0.4, 3, Uu)
    for k in range(5):
        np.testing.assert_array_equal(Uu2[k], Uu[k])
    c = math.sqrt(GAMMA * 0.9 / 1.3)
    expect_dt = 0.4 * (1.0 / n) / (0.4 + 0.2 + 0.1 + 3 * c)
    assert dts[0] == pytest.approx(expect_dt, rel=1e-14)


def test_rusanov_contact_wave_keeps_velocity_and_pressure():
    """A density variation advected at constant u and p: the Rusanov update
    keeps u and p constant (the flux is linear in rho along the contact)."""
    n = 8
    x = (np.arange(n) + 0.5) / n
    rho = np.broadcast_to(1.0 + 0.3 * np.sin(2 * np.pi * x)[None, None, :], (n, n, n)).reshape(-1).copy()
    V = [rho, np.full(n ** 3, 0.7), np.zeros(n ** 3), np.zeros(n ** 3), np.full(n ** 3, 1.0)]
    U = oracle.cons_from_prim(3, GAMMA, V)
    U2, _ = oracle.rusanov_run(n, GAMMA, 0.4, 4, U)
    V2 = oracle.prim_from_cons(3, GAMMA, U2)
    np.testing.assert_allclose(V2[1], 0.7, rtol=1e-13)
    np.testing.assert_allclose(V2[4], 1.0, rtol=1e-12)
    assert np.abs(V2[0] - rho).max() > 1e-3  # density did move


def test_rusanov_symmetries():
    n = 6
    U = _fv_init(n, seed=41, vel=0.0)
    V = oracle.prim_from_cons(3, GAMMA, U)
    Vs = [v.reshape(n, n, n) for v in V]  # [z, y, x]
    # give it a velocity field so all components are exercised
    Vs[1] = Vs[1] + 0.3 * np.sin(2 * np.pi * (np.arange(n) + 0.5) / n)[None, :, None]
    Vs[2] = Vs[2] - 0.2
    base = oracle.cons_from_prim(3, GAMMA, [v.reshape(-1) for v in Vs])
    out, _ = oracle.rusanov_run(n, GAMMA, 0.4, 2, base)
    # periodic translation along y
    sh = [np.roll(u.reshape(n, n, n), 2, axis=1).reshape(-1) for u in base]
    outs, _ = oracle.rusanov_run(n, GAMMA, 0.4, 2, sh)
    for k in range(5):
        np.testing.assert_allclose(outs[k], np.roll(out[k].reshape(n, n, n), 2, axis=1).reshape(-1),
                                   rtol=1e-13, atol=1e-13)
    # swap x and y axes (transpose grid, swap momentum components)
    def swap(Ul):
        g = [u.reshape(n, n, n).transpose(0, 2, 1).reshape(-1) for u in Ul]
        return [g[0], g[2], g[1], g[3], g[4]]
    outp, _ = oracle.rusanov_run(n, GAMMA, 0.4, 2, swap(base))
    ref = swap(out)
    for k in range(5):
        np.testing.assert_allclose(outp[k], ref[k], rtol=1e-12, atol=1e-13)


def test_rusanov_is_monotone_and_dissipative():
    """Under the CFL limit the Rusanov scheme is monotone: an advected density
    step creates no new extrema, and the density variance decays."""
    n = 8
    x = np.arange(n)
    step = np.where((x >= 2) & (x < 5), 2.0, 1.0)
    rho = np.broadcast_to(step[None, None, :], (n, n, n)).reshape(-1).copy()
    V = [rho, np.full(n ** 3, 0.5), np.zeros(n ** 3), np.zeros(n ** 3), np.full(n ** 3, 1.0)]
    U = oracle.cons_from_prim(3, GAMMA, V)
    var0 = rho.var()
    for steps in (1, 3):
        U2, _ = oracle.rusanov_run(n, GAMMA, 0.4, steps, U)
        r2 = U2[0]
        assert r2.max() <= 2.0 + 1e-12 and r2.min() >= 1.0 - 1e-12
        assert r2.var() < var0


# ---------------------------------------------------------------------------
# Roe flux and Roe-averaged characteristic transform
# ---------------------------------------------------------------------------

def _pair(n, D, seed):
    UL, _ = _rand_U(n, D, seed=seed)
    UR, _ = _rand_U(n, D, seed=seed + 1)
    return UL, UR


@pytest.mark.parametrize("D", [1, 2, 3])
def test_roe_flux_consistency(D):
    """Fh(U, U) = F(U): no dissipation between equal states."""
    U, _ = _rand_U(500, D, seed=51)
    for d in range(D):
        np.testing.assert_array_equal(_stack(oracle.roe_flux(D, d, GAMMA, U, U)),
                                      _stack(oracle.flux(D, d, GAMMA, U)))


@pytest.mark.parametrize("D", [1, 2, 3])
def test_roe_property(D):
    """Roe's matrix A^ = R^ Lambda^ L^ at the averaged state satisfies
    A^ (U_R - U_L) = F(U_R) - F(U_L) for the ideal gas; with the Roe flux this
    reads Fh = F(U_L) + sum_{lambda<0} ... , equivalently
    F(U_R) - F(U_L) = 2 (Fh - F(U_L)) + sum |lambda| alpha r - ... ; tested as
    (F_L + F_R)/2 - Fh = 1/2 sum |lambda^| alpha r with A^ dU = F_R - F_L."""
    UL, UR = _pair(800, D, 61)
    nv = D + 2
    dU = _stack(UR) - _stack(UL)
    for d in range(D):
        FL = _stack(oracle.flux(D, d, GAMMA, UL))
        FR = _stack(oracle.flux(D, d, GAMMA, UR))
        # Roe-averaged eigen-decomposition through the characteristic transform
        # at the Roe state: alpha = L^ dU, A^ dU = R^ (lambda^ * alpha)
        alpha = _stack(oracle.roe_char_transform(D, d, GAMMA, UL, UR, [dU[:, k] for k in range(nv)]))
        # eigenvalues of A^: u^ - c^, u^, u^ + c^ from the Roe state via R^ applied to unit vectors
        Rm = np.stack([_stack(oracle.roe_char_transform(D, d, GAMMA, UL, UR,
                                                          [np.full(dU.shape[0], float(k == j)) for k in range(nv)],
                                                          inverse=True)) for j in range(nv)], axis=-1)
        # u^ and c^: R^ columns r_1 = (1, v - c e_d, .) and r_nv = (1, v + c e_d, .)
        u_hat = 0.5 * (Rm[:, 1 + d, 0] + Rm[:, 1 + d, nv - 1])
        c_hat = 0.5 * (Rm[:, 1 + d, nv - 1] - Rm[:, 1 + d, 0])
        lam = np.stack([u_hat - c_hat] + [u_hat] * (nv - 2) + [u_hat + c_hat], axis=-1)
        AdU = np.einsum("nij,nj->ni", Rm, lam * alpha)
        scale = np.abs(FL) + np.abs(FR) + 1.0
        assert np.all(np.abs(AdU - (FR - FL)) <= 1e-10 * scale), d
        # and the flux itself
        Fh = _stack(oracle.roe_flux(D, d, GAMMA, UL, UR))
        diss = np.einsum("nij,nj->ni", Rm, np.abs(lam) * alpha)
        np.testing.assert_allclose(Fh, 0.5 * (FL + FR) - 0.5 * diss, rtol=1e-12, atol=1e-10)


def test_roe_average_of_equal_states_is_the_state():
    U, _ = _rand_U(300, 3, seed=71)
    W = synth.char_weights(300)
    for d in range(3):
        for inv in (False, True):
            np.testing.assert_allclose(_stack(oracle.roe_char_transform(3, d, GAMMA, U, U, W, inverse=inv)),
                                       _stack(oracle.char_transform(3, d, GAMMA, U, W, inverse=inv)),
                                       rtol=1e-13, atol=1e-13)


def test_roe_flux_upwinds_supersonic_flow():
    """All Roe eigenvalues positive (flow at Mach ~5 along x on both sides):
    the Roe flux is the left state's flux."""
    n = 400
    VL = synth.euler3d(n, seed=81)
    VR = synth.euler3d(n, seed=82)
    for V in (VL, VR):
        V[0][:] = 1.0 + 0.2 * (V[0] / 10.0)
        V[4][:] = 1.0 + 0.2 * (V[4] / 10.0)
        V[1][:] = 8.0
        V[2][:] = 0.1 * V[2]
        V[3][:] = 0.1 * V[3]
    UL = oracle.cons_from_prim(3, GAMMA, VL)
    UR = oracle.cons_from_prim(3, GAMMA, VR)
    Fh = _stack(oracle.roe_flux(3, 0, GAMMA, UL, UR))
    FL = _stack(oracle.flux(3, 0, GAMMA, UL))
    np.testing.assert_allclose(Fh, FL, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# primitive-variable forms and temperature
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_flux_from_primitives_is_the_flux(D):
    U, V = _rand_U(1500, D, seed=91)
    Vp = oracle.prim_from_cons(D, GAMMA, U)
    for d in [-1, *range(D)]:
        np.testing.assert_allclose(_stack(oracle.flux_prim(D, d, GAMMA, Vp)), _stack(oracle.flux(D, d, GAMMA, U)),
                                   rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_primitive_jacobian_chain_rule_and_differences(D):
    """dF/dV = A(U) dU/dV with dU/dV of U = (rho, rho v, p/(gamma-1) + rho|v|^2/2);
    and central differences of the primitive flux."""
    U, V = _rand_U(400, D, seed=93)
    V = oracle.prim_from_cons(D, GAMMA, U)
    nv = D + 2
    n = V[0].shape[0]
    rho = V[0]
    v = np.stack(V[1:D + 1], -1)
    dUdV = np.zeros((n, nv, nv))
    dUdV[:, 0, 0] = 1.0
    for i in range(D):
        dUdV[:, 1 + i, 0] = v[:, i]
        dUdV[:, 1 + i, 1 + i] = rho
        dUdV[:, nv - 1, 1 + i] = rho * v[:, i]
    dUdV[:, nv - 1, 0] = 0.5 * (v ** 2).sum(-1)
    dUdV[:, nv - 1, nv - 1] = 1.0 / (GAMMA - 1.0)
    for d in range(D):
        B = _stack(oracle.flux_jac_prim(D, d, GAMMA, V)).reshape(-1, nv, nv)
        A = _stack(oracle.flux_jac(D, d, GAMMA, U)).reshape(-1, nv, nv)
        np.testing.assert_allclose(B, A @ dUdV, rtol=1e-11, atol=1e-11)
        for j in range(nv):
            h = 1e-6 * np.maximum(1.0, np.abs(V[j]))
            Vp = [x.copy() for x in V]
            Vm = [x.copy() for x in V]
            Vp[j] += h
            Vm[j] -= h
            fd = (_stack(oracle.flux_prim(D, d, GAMMA, Vp)) - _stack(oracle.flux_prim(D, d, GAMMA, Vm))) / (2 * h)[:, None]
            assert np.all(np.abs(fd - B[:, :, j]) <= 1e-6 * (np.abs(B).max(axis=(1, 2))[:, None] + 1.0))


@pytest.mark.parametrize("D", [1, 3])
def test_temperature_is_the_ideal_gas_law(D):
    """With the paper's c_p = 7/2, c_v = 5/2 (gamma = 7/5, R = c_p - c_v = 1):
    p = rho R T, i.e. T = p / rho; for another c_v, T scales as 1/c_v."""
    U, V = _rand_U(1000, D, seed=95)
    T = oracle.temperature(D, GAMMA, 2.5, U)[0]
    np.testing.assert_allclose(T, V[D + 1] / V[0], rtol=1e-13)
    T2 = oracle.temperature(D, GAMMA, 5.0, U)[0]
    np.testing.assert_allclose(T2, 0.5 * T, rtol=1e-15)


# ---------------------------------------------------------------------------
# Rusanov step: hand-derived values of one step on a 4-cell contact
# ---------------------------------------------------------------------------

RUSANOV_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rusanov_contact_step.txt")


def _rusanov_golden():
    cases = {}
    with open(RUSANOV_GOLDEN) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cases[tok[1]] = {"u": float(tok[2]), "rho": {}}
            elif tok[1] == "dt":
                cases[tok[0]]["dt"] = _eval(tok[2])
            else:
                cases[tok[0]]["rho"][int(tok[2])] = _eval(tok[3])
    return cases


def contact_state(n, axis, u, levels=(1.0, 1.0, 4.0, 4.0)):
    """Conservative planes of the contact of the golden file along `axis`
    (0 = x, the fastest index; 1 = y; 2 = z), n = len(levels): rho by the
    cell's coordinate along the axis, p = 1, velocity u along the axis."""
    coord = np.indices((n, n, n))[2 - axis].reshape(-1)  # [z, y, x] layout
    rho = np.asarray(levels, dtype=np.float64)[coord]
    zero = np.zeros(n ** 3)
    V = [rho, zero.copy(), zero.copy(), zero.copy(), np.ones(n ** 3)]
    V[1 + axis] = np.full(n ** 3, u)
    return oracle.cons_from_prim(3, GAMMA, V), coord


@pytest.mark.parametrize("axis", [0, 1, 2], ids=["x", "y", "z"])
def test_rusanov_step_hand_values(axis):
    """One step of the oracle's scheme reproduces the hand-derived densities,
    time step, momentum u rho' and energy 2.5 + u^2 rho'/2 of
    tests/golden/rusanov_contact_step.txt along every axis.  The density moves
    by (dt/dx) times the face-flux difference, so a time step taken as dt
    instead of dt/dx (4x too small here), a sign slip in the dissipation or a
    face speed taken from the wrong side fails it."""
    n = 4
    cases = _rusanov_golden()
    assert set(cases) == {"rest", "right", "left"}
    for name, cs in cases.items():
        u = cs["u"]
        U, coord = contact_state(n, axis, u)
        U2, dts = oracle.rusanov_run(n, GAMMA, 0.4, 1, U)
        assert dts[0] == pytest.approx(cs["dt"], rel=1e-14), name
        assert oracle.rusanov_dt(n, GAMMA, 0.4, U) == pytest.approx(cs["dt"], rel=1e-14)
        want = np.array([cs["rho"][i] for i in range(n)])[coord]
        np.testing.assert_allclose(U2[0], want, rtol=1e-14, err_msg=name)
        np.testing.assert_allclose(U2[1 + axis], u * want, rtol=1e-14, atol=1e-15, err_msg=name)
        for k in range(3):
            if k != axis:
                np.testing.assert_array_equal(U2[1 + k], 0.0)
        np.testing.assert_allclose(U2[4], 2.5 + 0.5 * u * u * want, rtol=1e-14, err_msg=name)
        # rusanov_step with the golden dt gives the same state
        U3 = oracle.rusanov_step(n, GAMMA, cs["dt"], U)
        np.testing.assert_allclose(U3[0], want, rtol=1e-14, err_msg=name)
