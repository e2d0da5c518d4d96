"""GPU parity of the general-EOS blocks (fdbb_*_eos) against the FP64 CPU oracle.

Two equations of state stand in for a user EOS (paper section 2.2,
"Equations of state"): the Noble-Abel stiffened gas and the van der Waals
gas, on the workload ``synth.euler_eos``.  FP64 storage: |gpu - oracle| <=
1e-12 * S (S the oracle's running-error scale; S == 0 only for exact copies,
which must be bit-equal).  FP64 storage in double-word arithmetic
meets the same FP64 bound.  FP32 / FP16 / BF16 storage (float arithmetic):
the oracle runs on the dequantised inputs and |gpu - oracle| <= u_store
|oracle| + (half the storage type's subnormal spacing) + 64 * 2^-24 * S, u_store
the unit roundoff of the storage type.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1809_09851_gb300 import blocks, capi, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
MODELS = [synth.EOS_NASG, synth.EOS_VDW]
IDS = ["nasg", "vdw"]
SIZES = [1, 7, 513, 65539]
# storage / arithmetic forms: (dtype, double-word)
FORMS = {"f64": (torch.float64, False), "f64dw": (torch.float64, True), "f32": (torch.float32, False),
         "f16": (torch.float16, False), "bf16": (torch.bfloat16, False)}
U_STORE = {torch.float64: 0.0, torch.float32: 2.0 ** -24, torch.float16: 2.0 ** -11, torch.bfloat16: 2.0 ** -8}
# half the subnormal spacing of the storage type (rounding below its smallest normal number)
TINY_STORE = {torch.float64: 0.0, torch.float32: 2.0 ** -150, torch.float16: 2.0 ** -25,
              torch.bfloat16: 2.0 ** -134}
TOL = {torch.float64: 1e-12, torch.float32: 64 * 2.0 ** -24, torch.float16: 64 * 2.0 ** -24,
       torch.bfloat16: 64 * 2.0 ** -24}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_09851_gb300 import build
    build.build()
    capi.lib()
    assert torch.cuda.is_available()


def dev(planes, dtype):
    """numpy planes -> device tensors of `dtype` and their dequantised float64 values."""
    t = [torch.from_numpy(np.ascontiguousarray(p)).to(DEV).to(dtype) for p in planes]
    return t, [x.double().cpu().numpy() for x in t]


def host(planes):
    return [t.double().cpu().numpy() for t in planes]


def check(got, ref, S, dtype, what):
    assert len(got) == len(ref), what
    for c, (g, o, s) in enumerate(zip(got, ref, S)):
        bound = U_STORE[dtype] * np.abs(o) + TINY_STORE[dtype] + TOL[dtype] * s
        ok = np.abs(g - o) <= bound
        if not ok.all():
            i = int(np.argmin(ok))
            raise AssertionError(f"{what}: plane {c} point {i}: gpu={g[i]!r} oracle={o[i]!r} S={s[i]!r}")


def case(eos, n, D, dtype, seed=1809):
    V = synth.euler_eos(n, D, seed=seed)
    U = oracle.eos_cons_from_prim(eos, D, V)
    W = synth.char_weights(n, D + 2, seed=seed + 1)
    G = synth.cotangent(n, D + 2, seed=seed + 2)
    Ud, U = dev(U, dtype)
    Vd, V = dev(V, dtype)
    Wd, W = dev(W, dtype)
    Gd, G = dev(G, dtype)
    return (U, V, W, G), (Ud, Vd, Wd, Gd)


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_pointwise_state_blocks(D, n, eos, form):
    dtype, dw = FORMS[form]
    (U, V, W, G), (Ud, Vd, Wd, Gd) = case(eos, n, D, dtype)
    ref, S = oracle.eos_prim_from_cons(eos, D, U, scale=True)
    check(host(blocks.prim_from_cons_eos(Ud, eos, dw=dw)), ref, S, dtype, "prim_from_cons")
    ref, S = oracle.eos_cons_from_prim(eos, D, V, scale=True)
    check(host(blocks.cons_from_prim_eos(Vd, eos, dw=dw)), ref, S, dtype, "cons_from_prim")
    ref, S = oracle.eos_pc(eos, D, U, scale=True)
    check(host(blocks.pressure_eos(Ud, eos, dw=dw)), ref, S, dtype, "p, c")
    ref, S = oracle.eos_temperature(eos, D, U, scale=True)
    check(host([blocks.temperature_eos(Ud, eos, dw=dw)]), ref, S, dtype, "T")
    ref, S = oracle.eos_flux(eos, D, -1, U, scale=True)
    check(host(blocks.flux_eos(Ud, eos, -1, dw=dw)), ref, S, dtype, "flux all")
    ref, S = oracle.eos_flux_prim(eos, D, -1, V, scale=True)
    check(host(blocks.flux_prim_eos(Vd, eos, -1, dw=dw)), ref, S, dtype, "flux_prim all")


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("eos", MODELS, ids=IDS)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_directional_blocks(D, n, eos, form):
    dtype, dw = FORMS[form]
    (U, V, W, G), (Ud, Vd, Wd, Gd) = case(eos, n, D, dtype)
    for d in range(D):
        ref, S = oracle.eos_flux(eos, D, d, U, scale=True)
        check(host(blocks.flux_eos(Ud, eos, d, dw=dw)), ref, S, dtype, f"flux {d}")
        ref, S = oracle.eos_flux_jac(eos, D, d, U, scale=True)
        check(host(blocks.flux_jac_eos(Ud, eos, d, dw=dw)), ref, S, dtype, f"flux_jac {d}")
        for inv in (False, True):
            ref, S = oracle.eos_char_transform(eos, D, d, U, W, inverse=inv, scale=True)
            check(host(blocks.char_transform_eos(Ud, Wd, eos, d, inverse=inv, dw=dw)), ref, S, dtype,
                  f"char {'inv' if inv else 'fwd'} {d}")
        ref, S = oracle.eos_flux_vjp(eos, D, d, U, G, scale=True)
        check(host(blocks.flux_vjp_eos(Ud, Gd, eos, d, dw=dw)), ref, S, dtype, f"vjp {d}")
        ref, S = oracle.eos_euler_fused(eos, D, d, U, W, scale=True)
        F, A, Y = blocks.euler_fused_eos(Ud, Wd, eos, d, dw=dw)
        check(host(F + A + Y), ref, S, dtype, f"fused {d}")
        ref, S = oracle.eos_flux_prim(eos, D, d, V, scale=True)
        check(host(blocks.flux_prim_eos(Vd, eos, d, dw=dw)), ref, S, dtype, f"flux_prim {d}")
        ref, S = oracle.eos_flux_jac_prim(eos, D, d, V, scale=True)
        check(host(blocks.flux_jac_prim_eos(Vd, eos, d, dw=dw)), ref, S, dtype, f"flux_jac_prim {d}")


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("eos", MODELS, ids=IDS)
def test_fused_staged_path(eos, form):
    """Large enough for the staged (bulk-copy) kernel: >= 4 tiles per SM, plus a ragged tail."""
    dtype, dw = FORMS[form]
    n = (1 << 20) + 5
    (U, V, W, G), (Ud, Vd, Wd, Gd) = case(eos, n, 3, dtype, seed=77)
    ref, S = oracle.eos_euler_fused(eos, 3, 0, U, W, scale=True)
    F, A, Y = blocks.euler_fused_eos(Ud, Wd, eos, 0, dw=dw)
    check(host(F + A + Y), ref, S, dtype, "fused staged")
    assert capi.lib().fdbb_device_status() == 0


def test_double_word_out_of_range_points_and_parameters():
    """Points outside the double-word range (tiny densities and pressures) are
    recomputed in IEEE double; parameters outside it make the whole call IEEE
    double.  Both meet the FP64 bound."""
    n = 20000
    for eos in (synth.EOS_NASG, dict(synth.EOS_NASG, p_inf=1e-9), dict(synth.EOS_VDW, a=3e-8)):
        V = synth.euler_eos(n, 3, seed=91)
        V[0][::7] *= 1e-9  # rho ~ 1e-9: outside [2^-24, 2^24]
        if eos["kind"] == "nasg":
            V[4][::5] *= 1e-9  # p ~ 1e-9 (p + p_inf stays positive)
        U = oracle.eos_cons_from_prim(eos, 3, V)
        W = synth.char_weights(n, 5, seed=92)
        Ud, U = dev(U, torch.float64)
        Wd, W = dev(W, torch.float64)
        ref, S = oracle.eos_euler_fused(eos, 3, 1, U, W, scale=True)
        F, A, Y = blocks.euler_fused_eos(Ud, Wd, eos, 1, dw=True)
        check(host(F + A + Y), ref, S, torch.float64, f"fused dw {eos}")


def test_exact_copies_and_skipped_outputs():
    eos = synth.EOS_NASG
    (U, V, W, G), (Ud, Vd, Wd, Gd) = case(eos, 4099, 3, torch.float64)
    F, A, Y = blocks.euler_fused_eos(Ud, Wd, eos, 1)
    for d in range(3):
        assert torch.equal(F[5 * d], Ud[1 + d])  # F_d[0] = m_d, bit for bit
    # skip F and Y: W is not needed
    _, A2, _ = blocks.euler_fused_eos(Ud, None, eos, 1, out=(None, [torch.empty_like(Ud[0]) for _ in range(25)], None))
    for a, b in zip(A, A2):
        assert torch.equal(a, b)
    # only c from the pressure block
    p, c = blocks.pressure_eos(Ud, eos, want_p=False)
    assert p is None
    _, c_ref = blocks.pressure_eos(Ud, eos)
    assert torch.equal(c, c_ref)
    # rho onto itself is not copied
    Vout = [Ud[0]] + [torch.empty_like(Ud[0]) for _ in range(4)]
    blocks.prim_from_cons_eos(Ud, eos, out=Vout)
    assert torch.equal(Vout[0], Ud[0])


def test_ideal_kind_forwards_and_unstiffened_nasg_matches_ideal():
    """kind "ideal" runs the ideal-gas kernels (bit-equal results); NASG with
    p_inf = b = q = 0 is the ideal gas through the general kernels (equal
    within the FP64 bound of the ideal-gas oracle)."""
    D, n, g = 3, 20001, 1.4
    V = synth.euler3d(n, seed=5)
    U = oracle.cons_from_prim(D, g, V)
    W = synth.char_weights(n, 5)
    Ud, U = dev(U, torch.float64)
    Wd, W = dev(W, torch.float64)
    ideal = {"kind": "ideal", "gamma": g}
    a = blocks.euler_fused_eos(Ud, Wd, ideal, 2)
    b = blocks.euler_fused(Ud, Wd, 2, g)
    for x, y in zip(a[0] + a[1] + a[2], b[0] + b[1] + b[2]):
        assert torch.equal(x, y)
    for dt in (torch.float16, torch.bfloat16):  # the ideal kind keeps every storage type
        Uh = [t.to(dt) for t in Ud]
        assert torch.equal(blocks.flux_eos(Uh, ideal, 0)[4], blocks.flux(Uh, 0, g)[4])
    nasg0 = {"kind": "nasg", "gamma": g, "cv": 2.5}
    ref, S = oracle.euler_fused(D, 2, g, U, W, scale=True)
    F, A, Y = blocks.euler_fused_eos(Ud, Wd, nasg0, 2)
    check(host(F + A + Y), ref, S, torch.float64, "nasg0 fused")
    ref, S = oracle.temperature(D, g, 2.5, U, scale=True)
    check(host([blocks.temperature_eos(Ud, nasg0)]), ref, S, torch.float64, "nasg0 T")


def test_empty_and_rejected_dtypes():
    eos = synth.EOS_VDW
    # n == 0 through the C ABI: validated, nothing launched, outputs untouched
    U = [torch.ones(8, dtype=torch.float64, device=DEV) for _ in range(5)]
    F = [torch.full((8,), 7.0, dtype=torch.float64, device=DEV) for _ in range(15)]
    m = capi.eos_model(eos)
    st = capi.lib().fdbb_flux_eos(ctypes.byref(m), 3, -1, 0, capi.FDBB_F64, capi.planes([t.data_ptr() for t in U]),
                                  capi.planes([t.data_ptr() for t in F]), None)
    torch.cuda.synchronize()
    assert st == 0 and all(bool((f == 7.0).all()) for f in F)
    # an unknown storage type is refused before any launch
    st = capi.lib().fdbb_flux_eos(ctypes.byref(m), 3, 0, 8, 9, capi.planes([t.data_ptr() for t in U]),
                                  capi.planes([t.data_ptr() for t in F[:5]]), None)
    assert st == 4


@pytest.mark.slow
@pytest.mark.parametrize("form", ["f64dw", "f64", "f32"])
def test_full_size_fused_sampled(form):
    """The fused pass under NASG at the benchmark size (N = 2^26, the
    general-EOS leg's launch configuration): sampled points against the oracle."""
    dtype, dw = FORMS[form]
    eos = synth.EOS_NASG
    n = 1 << 26
    V = synth.euler_eos(n, 3)
    U = oracle.eos_cons_from_prim(eos, 3, V)
    W = synth.char_weights(n, 5)
    del V
    Ud, U = dev(U, dtype)
    Wd, W = dev(W, dtype)
    F, A, Y = blocks.euler_fused_eos(Ud, Wd, eos, 0, dw=dw)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([rng.integers(0, n, 4096), np.arange(n - 37, n), np.arange(5)]))
    it = torch.from_numpy(idx).to(DEV)
    got = [t[it].double().cpu().numpy() for t in (*F, *A, *Y)]
    ref, S = oracle.eos_euler_fused(eos, 3, 0, [u[idx] for u in U], [w[idx] for w in W], scale=True)
    check(got, ref, S, dtype, "full-size fused nasg")
