"""Pins of the oracle's general-EOS blocks against facts it does not compute itself.

The general-EOS oracle (paper section 2.2, "Equations of state") is checked
against: the already pinned ideal-gas oracle (NASG with p_inf = b = q = 0 is
the ideal gas), closed forms of the sound speed and the thermal equation of
state from the literature, central finite differences of p(rho, e),
rho e(rho, p) and of the fluxes, thermodynamic integrability of (p, T),
identities of the eigen-structure (L R = I, A R = R Lambda, numpy inverse),
and round trips.  A dropped term, a wrong sign or a swapped derivative in any
EOS formula or in the general Jacobian / eigenvectors fails one of them.
"""
import numpy as np
import pytest

import oracle
from paper_1809_09851_gb300 import synth

NASG = synth.EOS_NASG
VDW = synth.EOS_VDW
MODELS = [NASG, VDW]
IDS = ["nasg", "vdw"]


def _stack(planes):
    return np.stack(planes, axis=-1)


def _U(eos, n, D, seed=3):
    V = synth.euler_eos(n, D, seed=seed)
    return oracle.eos_cons_from_prim(eos, D, V), V


def _close(a, b, S, tol):
    a, b, S = np.asarray(a), np.asarray(b), np.asarray(S)
    assert np.all(np.abs(a - b) <= tol * S), float(np.max(np.abs(a - b) / np.maximum(S, 1e-300)))


# ---------------------------------------------------------------------------
# reduction to the ideal gas
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [1, 2, 3])
def test_nasg_without_stiffening_is_the_ideal_gas(D):
    g, cv = 1.4, 2.5
    ideal = {"kind": "nasg", "gamma": g, "cv": cv}
    V = synth.euler3d(700, seed=17, D=D) if D > 1 else synth.euler1d(700, seed=17)
    U = oracle.cons_from_prim(D, g, V)
    n = V[0].shape[0]
    nv = D + 2
    W = synth.char_weights(n, nv)
    G = synth.cotangent(n, nv)
    tol = 64 * 2.0 ** -53

    def same(gen, ref):
        (o, s) = gen
        (r, t) = ref
        for k in range(len(o)):
            _close(o[k], r[k], s[k] + t[k], tol)

    same(oracle.eos_cons_from_prim(ideal, D, V, scale=True), oracle.cons_from_prim(D, g, V, scale=True))
    same(oracle.eos_prim_from_cons(ideal, D, U, scale=True), oracle.prim_from_cons(D, g, U, scale=True))
    same(oracle.eos_pc(ideal, D, U, scale=True), oracle.eos(D, g, U, scale=True))
    same(oracle.eos_temperature(ideal, D, U, scale=True), oracle.temperature(D, g, cv, U, scale=True))
    for d in [-1, *range(D)]:
        same(oracle.eos_flux(ideal, D, d, U, scale=True), oracle.flux(D, d, g, U, scale=True))
        same(oracle.eos_flux_prim(ideal, D, d, V, scale=True), oracle.flux_prim(D, d, g, V, scale=True))
    for d in range(D):
        same(oracle.eos_flux_jac(ideal, D, d, U, scale=True), oracle.flux_jac(D, d, g, U, scale=True))
        same(oracle.eos_flux_jac_prim(ideal, D, d, V, scale=True), oracle.flux_jac_prim(D, d, g, V, scale=True))
        for inv in (False, True):
            same(oracle.eos_char_transform(ideal, D, d, U, W, inverse=inv, scale=True),
                 oracle.char_transform(D, d, g, U, W, inverse=inv, scale=True))
        same(oracle.eos_flux_vjp(ideal, D, d, U, G, scale=True), oracle.flux_vjp(D, d, g, U, G, scale=True))
        same(oracle.eos_euler_fused(ideal, D, d, U, W, scale=True), oracle.euler_fused(D, d, g, U, W, scale=True))


# ---------------------------------------------------------------------------
# the EOS functions themselves
# ---------------------------------------------------------------------------

def _rho_e(eos, n=4000, seed=5):
    """(rho, e) on the workload's range: e from p through the oracle's inverse."""
    V = synth.euler_eos(n, 1, seed=seed)
    rho, p = V[0], V[2]
    z, _ = oracle.eos_point(eos, rho, p)[1][0], None
    return rho, z / rho, p


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
def test_inverse_recovers_the_pressure(eos):
    rho, e, p = _rho_e(eos)
    (pp, _, _, _), _ = oracle.eos_point(eos, rho, e)
    np.testing.assert_allclose(pp, p, rtol=1e-12, atol=1e-12)


def test_closed_forms_of_sound_speed_and_thermal_law():
    """NASG: c^2 = gamma (p + p_inf) / (rho (1 - b rho)),
    p = (gamma - 1) c_v rho T / (1 - b rho) - p_inf;
    van der Waals: c^2 = gamma (p + a rho^2) / (rho (1 - b rho)) - 2 a rho,
    p = (gamma - 1) c_v rho T / (1 - b rho) - a rho^2."""
    for eos in MODELS:
        D = 2
        U, V = _U(eos, 3000, D, seed=21)
        p, c = oracle.eos_pc(eos, D, U)
        T = oracle.eos_temperature(eos, D, U)[0]
        rho = V[0]
        g, b, cv = eos["gamma"], eos.get("b", 0.0), eos["cv"]
        if eos["kind"] == "nasg":
            c2 = g * (p + eos["p_inf"]) / (rho * (1 - b * rho))
            p_th = (g - 1) * cv * rho * T / (1 - b * rho) - eos["p_inf"]
        else:
            a = eos["a"]
            c2 = g * (p + a * rho ** 2) / (rho * (1 - b * rho)) - 2 * a * rho
            p_th = (g - 1) * cv * rho * T / (1 - b * rho) - a * rho ** 2
        np.testing.assert_allclose(c ** 2, c2, rtol=1e-11)
        np.testing.assert_allclose(p_th, V[D + 1], rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(p, V[D + 1], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
def test_partial_derivatives_central_differences(eos):
    rho, e, p = _rho_e(eos, n=2000, seed=7)
    (P, p_rho, p_e, _), _ = oracle.eos_point(eos, rho, e)
    h = 1e-6
    (Pp, _, _, _), _ = oracle.eos_point(eos, rho * (1 + h), e)
    (Pm, _, _, _), _ = oracle.eos_point(eos, rho * (1 - h), e)
    np.testing.assert_allclose((Pp - Pm) / (2 * h * rho), p_rho, rtol=1e-6, atol=1e-7)
    he = h * np.maximum(1.0, np.abs(e))
    (Pp, _, _, _), _ = oracle.eos_point(eos, rho, e + he)
    (Pm, _, _, _), _ = oracle.eos_point(eos, rho, e - he)
    np.testing.assert_allclose((Pp - Pm) / (2 * he), p_e, rtol=1e-6, atol=1e-7)
    # rho e(rho, p): derivatives in rho at constant p and in p at constant rho
    _, (z, z_rho, z_p) = oracle.eos_point(eos, rho, p)
    _, (zp, _, _) = oracle.eos_point(eos, rho * (1 + h), p)
    _, (zm, _, _) = oracle.eos_point(eos, rho * (1 - h), p)
    np.testing.assert_allclose((zp - zm) / (2 * h * rho), z_rho, rtol=1e-6, atol=1e-7)
    _, (zp, _, _) = oracle.eos_point(eos, rho, p * (1 + h))
    _, (zm, _, _) = oracle.eos_point(eos, rho, p * (1 - h))
    np.testing.assert_allclose((zp - zm) / (2 * h * p), z_p, rtol=1e-6, atol=1e-7)
    # implicit-function relations between the two sets
    np.testing.assert_allclose(z_p, rho / p_e, rtol=1e-12)
    np.testing.assert_allclose(z_rho, e - rho * p_rho / p_e, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
def test_sound_speed_is_the_isentropic_derivative(eos):
    """c^2 = dp/drho along de = p / rho^2 drho (second-order central difference)."""
    D = 1
    U, V = _U(eos, 2000, D, seed=23)
    p, c = oracle.eos_pc(eos, D, U)
    rho = V[0]
    e = oracle.eos_point(eos, rho, p)[1][0] / rho
    h = 1e-5 * rho
    # second-order isentrope through (rho, e): e(rho + dr) = e + p/rho^2 dr + O(dr^2);
    # the O(dr^2) term is symmetric and cancels in the central difference.
    (Pp, _, _, _), _ = oracle.eos_point(eos, rho + h, e + p / rho ** 2 * h)
    (Pm, _, _, _), _ = oracle.eos_point(eos, rho - h, e - p / rho ** 2 * h)
    np.testing.assert_allclose((Pp - Pm) / (2 * h), c ** 2, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
def test_temperature_is_thermodynamically_consistent(eos):
    """An entropy s(v, e) with ds = (de + p dv) / T exists iff
    d(1/T)/dv |_e = d(p/T)/de |_v  (v = 1/rho), checked by central differences."""
    rho, e, _ = _rho_e(eos, n=2000, seed=9)
    v = 1.0 / rho

    def inv_T(vv, ee):
        return 1.0 / oracle.eos_point(eos, 1.0 / vv, ee)[0][3]

    def p_T(vv, ee):
        out = oracle.eos_point(eos, 1.0 / vv, ee)[0]
        return out[0] / out[3]

    hv, he = 1e-5 * v, 1e-5 * np.maximum(1.0, np.abs(e))
    lhs = (inv_T(v + hv, e) - inv_T(v - hv, e)) / (2 * hv)
    rhs = (p_T(v, e + he) - p_T(v, e - he)) / (2 * he)
    scale = np.abs(lhs) + np.abs(rhs) + np.abs(inv_T(v, e)) / v
    assert np.all(np.abs(lhs - rhs) <= 1e-6 * scale)
    # and a wrong temperature law (T off by a density-dependent factor) fails it
    def inv_T_bad(vv, ee):
        return (1.0 + 0.1 / vv) / oracle.eos_point(eos, 1.0 / vv, ee)[0][3]
    bad = (inv_T_bad(v + hv, e) - inv_T_bad(v - hv, e)) / (2 * hv)
    assert np.any(np.abs(bad - rhs) > 1e-3 * scale)


# ---------------------------------------------------------------------------
# blocks under a general EOS
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_cons_prim_round_trip(eos, D):
    U, V = _U(eos, 1500, D, seed=25)
    back = oracle.eos_prim_from_cons(eos, D, U)
    for k in range(D + 2):
        np.testing.assert_allclose(back[k], V[k], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_flux_definition(eos, D):
    """F_d = (m_d, m_d v + p e_d, v_d (rhoE + p)) with p from the EOS block."""
    U, V = _U(eos, 1000, D, seed=27)
    p = oracle.eos_pc(eos, D, U)[0]
    nv = D + 2
    F_all = oracle.eos_flux(eos, D, -1, U)
    for d in range(D):
        F = oracle.eos_flux(eos, D, d, U)
        u = U[1 + d] / U[0]
        np.testing.assert_array_equal(F[0], U[1 + d])
        for i in range(D):
            ref = U[1 + d] * U[1 + i] / U[0] + (p if i == d else 0.0)
            np.testing.assert_allclose(F[1 + i], ref, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(F[nv - 1], u * (U[nv - 1] + p), rtol=1e-12, atol=1e-13)
        for k in range(nv):
            np.testing.assert_array_equal(F_all[d * nv + k], F[k])


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_jacobian_central_differences(eos, D):
    U, _ = _U(eos, 256, D, seed=29)
    nv = D + 2
    for d in range(D):
        A = _stack(oracle.eos_flux_jac(eos, D, d, U)).reshape(-1, nv, nv)
        for j in range(nv):
            h = 1e-6 * np.maximum(1.0, np.abs(U[j]))
            Up = [u.copy() for u in U]
            Um = [u.copy() for u in U]
            Up[j] += h
            Um[j] -= h
            fd = (_stack(oracle.eos_flux(eos, D, d, Up)) - _stack(oracle.eos_flux(eos, D, d, Um))) / (2 * h)[:, None]
            scale = np.abs(A).max(axis=(1, 2))[:, None] + 1.0
            assert np.all(np.abs(fd - A[:, :, j]) <= 1e-6 * scale), (d, j)


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_eigenvectors(eos, D):
    U, V = _U(eos, 1024, D, seed=31)
    nv = D + 2
    I = np.eye(nv)
    c = oracle.eos_pc(eos, D, U)[1]
    for d in range(D):
        R, L, lam, aux = oracle.eos_eig(eos, D, d, U)
        R = _stack(R).reshape(-1, nv, nv)
        L = _stack(L).reshape(-1, nv, nv)
        lam = _stack(lam)
        A = _stack(oracle.eos_flux_jac(eos, D, d, U)).reshape(-1, nv, nv)
        np.testing.assert_allclose(L @ R, np.broadcast_to(I, L.shape), atol=1e-10)
        np.testing.assert_allclose(L, np.linalg.inv(R), rtol=1e-8, atol=1e-8)
        scale = np.abs(A) @ np.abs(R) + 1.0
        assert np.all(np.abs(A @ R - R * lam[:, None, :]) <= 1e-11 * scale)
        np.testing.assert_allclose(lam[:, 0], V[1 + d] - c, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(lam[:, -1], V[1 + d] + c, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_char_transform_vjp_and_fused(eos, D):
    U, _ = _U(eos, 600, D, seed=33)
    nv = D + 2
    n = U[0].shape[0]
    W = synth.char_weights(n, nv)
    G = synth.cotangent(n, nv)
    Ws = _stack(W)
    for d in range(D):
        R, L, lam, _ = oracle.eos_eig(eos, D, d, U)
        Rm = _stack(R).reshape(-1, nv, nv)
        # inverse = R W (numpy matmul); forward = R^{-1} W (numpy solve)
        Yi = _stack(oracle.eos_char_transform(eos, D, d, U, W, inverse=True))
        np.testing.assert_allclose(Yi, np.einsum("nij,nj->ni", Rm, Ws), rtol=1e-12, atol=1e-12)
        Yf = _stack(oracle.eos_char_transform(eos, D, d, U, W))
        np.testing.assert_allclose(Yf, np.linalg.solve(Rm, Ws[..., None])[..., 0], rtol=1e-8, atol=1e-8)
        # VJP = A^T G (numpy)
        A = _stack(oracle.eos_flux_jac(eos, D, d, U)).reshape(-1, nv, nv)
        gU = _stack(oracle.eos_flux_vjp(eos, D, d, U, G))
        np.testing.assert_allclose(gU, np.einsum("nji,nj->ni", A, _stack(G)), rtol=1e-11, atol=1e-11)
        # fused = fluxes, A_d, L_d W in that order
        out = oracle.eos_euler_fused(eos, D, d, U, W)
        ref = oracle.eos_flux(eos, D, -1, U) + oracle.eos_flux_jac(eos, D, d, U) + \
            oracle.eos_char_transform(eos, D, d, U, W)
        for a, b in zip(out, ref):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_primitive_forms(eos, D):
    """Flux from V equals the flux of U(V); dF/dV = A(U) dU/dV with dU/dV from
    central differences of the cons-from-prim block, and central differences
    of the primitive flux itself."""
    U, V = _U(eos, 300, D, seed=35)
    V = oracle.eos_prim_from_cons(eos, D, U)
    nv = D + 2
    for d in [-1, *range(D)]:
        np.testing.assert_allclose(_stack(oracle.eos_flux_prim(eos, D, d, V)), _stack(oracle.eos_flux(eos, D, d, U)),
                                   rtol=1e-11, atol=1e-11)
    dUdV = np.zeros((V[0].shape[0], nv, nv))
    for j in range(nv):
        h = 1e-6 * np.maximum(1.0, np.abs(V[j]))
        Vp = [x.copy() for x in V]
        Vm = [x.copy() for x in V]
        Vp[j] += h
        Vm[j] -= h
        dUdV[:, :, j] = (_stack(oracle.eos_cons_from_prim(eos, D, Vp)) -
                         _stack(oracle.eos_cons_from_prim(eos, D, Vm))) / (2 * h)[:, None]
    for d in range(D):
        B = _stack(oracle.eos_flux_jac_prim(eos, D, d, V)).reshape(-1, nv, nv)
        A = _stack(oracle.eos_flux_jac(eos, D, d, U)).reshape(-1, nv, nv)
        scale = np.abs(A) @ np.abs(dUdV) + 1.0
        assert np.all(np.abs(B - A @ dUdV) <= 1e-6 * scale)
        for j in range(nv):
            h = 1e-6 * np.maximum(1.0, np.abs(V[j]))
            Vp = [x.copy() for x in V]
            Vm = [x.copy() for x in V]
            Vp[j] += h
            Vm[j] -= h
            fd = (_stack(oracle.eos_flux_prim(eos, D, d, Vp)) - _stack(oracle.eos_flux_prim(eos, D, d, Vm))) \
                / (2 * h)[:, None]
            assert np.all(np.abs(fd - B[:, :, j]) <= 1e-6 * (np.abs(B).max(axis=(1, 2))[:, None] + 1.0))


def test_error_scale_bounds_value():
    """S >= |o|, except S = 0 where the output is exact: a copy of an input
    (F_d[0] = m_d) or a literal entry (0 or 1) of the Jacobian."""
    for eos in MODELS:
        U, _ = _U(eos, 500, 3, seed=37)
        out, S = oracle.eos_euler_fused(eos, 3, 0, U, synth.char_weights(500, 5), scale=True)
        for k, (o, s) in enumerate(zip(out, S)):
            exact = s == 0
            assert np.all(s[~exact] >= np.abs(o[~exact]) * (1 - 1e-15))
            if k in (0, 5, 10):
                assert exact.all()
                np.testing.assert_array_equal(o, U[1 + k // 5])
            elif exact.any():
                assert 15 <= k < 40 and np.all(np.isin(o[exact], (0.0, 1.0)))


def test_argument_checks():
    U, _ = _U(NASG, 8, 1)
    for bad in ({"kind": "nasg", "gamma": 1.0}, {"kind": "nasg", "gamma": 1.4, "b": -0.1},
                {"kind": "nasg", "gamma": 1.4, "p_inf": -1.0}, {"kind": "vdw", "gamma": 1.4, "a": -1.0},
                {"kind": "nasg", "gamma": 1.4, "cv": 0.0}):
        with pytest.raises(ValueError):
            oracle.eos_pc(bad, 1, U)
    with pytest.raises(KeyError):
        oracle.eos_pc({"kind": "ideal", "gamma": 1.4}, 1, U)
    with pytest.raises(ValueError):
        oracle.eos_flux(NASG, 1, 1, U)
