"""GPU parity: every entry point of the C ABI against the FP64 CPU oracle.

FP64 storage: |gpu - oracle| <= 1e-12 * S per output, S the oracle's
first-order running-error scale (S >= |oracle|, larger where the formula
cancels; S == 0 only for exact copies, which must then be bit-equal).
Reduced-precision storage (f32/f16/bf16, float arithmetic): the oracle runs on
the dequantised inputs and |gpu - oracle| <= u_store |oracle| + 64 * 2^-24 * S,
u_store the unit roundoff of the output storage type (plus half its
subnormal spacing, for results below its smallest normal number).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_09851_gb300 import blocks, capi, synth

pytestmark = pytest.mark.gpu

G = 1.4
SIZES = [1, 2, 7, 31, 513, 65539]  # ragged tails, several 256-thread tiles
U_STORE = {torch.float64: 0.0, torch.float32: 2.0 ** -24, torch.float16: 2.0 ** -11,
           torch.bfloat16: 2.0 ** -8}
# half the spacing of the storage type's subnormals: below its smallest normal
# number, rounding to the storage type is an absolute error of at most this
TINY_STORE = {torch.float64: 0.0, torch.float32: 2.0 ** -150, torch.float16: 2.0 ** -25,
              torch.bfloat16: 2.0 ** -134}
TOL_F64 = 1e-12
K_F32 = 64 * 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_09851_gb300 import build
    build.build()
    capi.lib()
    assert torch.cuda.is_available()


DEV = "cuda:0"


def sm_count() -> int:
    return torch.cuda.get_device_properties(DEV).multi_processor_count


def staged_n(tile: int, tail: int) -> int:
    """A size at which every SM gets at least four tiles of `tile` points (the
    staged kernel's threshold), plus a ragged tail."""
    return 4 * sm_count() * tile + tail


def assert_staged():
    info = capi.last_launch()
    assert info.kernel == capi.FDBB_KERNEL_STAGED, (info.kernel, info.grid, info.points_per_thread)


def fields(n, D, seed=1809):
    V = synth.euler3d(n, seed=seed, D=D) if D > 1 else synth.euler1d(n, seed=seed)
    U = oracle.cons_from_prim(D, G, V)
    W = synth.char_weights(n, D + 2, seed=seed + 1)
    return V, U, W


def quantise(planes, dtype):
    """Round float64 numpy planes to `dtype`; returns (device tensors, dequantised float64)."""
    dev = [torch.from_numpy(np.ascontiguousarray(p)).to(DEV).to(dtype) for p in planes]
    back = [t.double().cpu().numpy() for t in dev]
    return dev, back


def host(planes):
    return [t.double().cpu().numpy() for t in planes]


def check(got, ref, S, dtype, what):
    u_out = U_STORE[dtype]
    k = TOL_F64 if dtype == torch.float64 else K_F32
    assert len(got) == len(ref)
    for c, (g, o, s) in enumerate(zip(got, ref, S)):
        bound = u_out * np.abs(o) + TINY_STORE[dtype] + k * s
        err = np.abs(g - o)
        ok = err <= bound
        # a stored state that is non-physical (p < 0 once rounded to 16 bits):
        # the output is undefined, NaN in the oracle on the same inputs
        ok |= np.isnan(o) & (np.isnan(g) | (dtype != torch.float64))
        if dtype == torch.float16:
            ok |= np.abs(o) > 6.0e4  # beyond the f16 range the stored value is inf
        if not ok.all():
            i = int(np.argmin(ok))
            raise AssertionError(f"{what}: plane {c} point {i}: gpu={g[i]!r} oracle={o[i]!r} "
                                 f"S={s[i]!r} bound={bound[i]!r}")


# ---------------------------------------------------------------------------
# FP64, every block, every dim / dir, several sizes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dw", [False, True], ids=["f64", "f64dw"])
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_f64_variables_and_eos(n, D, dw):
    V, U, W = fields(n, D)
    Ud, _ = quantise(U, torch.float64)
    Vd, _ = quantise(V, torch.float64)
    ref, S = oracle.prim_from_cons(D, G, U, scale=True)
    check(host(blocks.prim_from_cons(Ud, G, dw=dw)), ref, S, torch.float64, "prim_from_cons")
    ref, S = oracle.cons_from_prim(D, G, V, scale=True)
    check(host(blocks.cons_from_prim(Vd, G, dw=dw)), ref, S, torch.float64, "cons_from_prim")
    ref, S = oracle.eos(D, G, U, scale=True)
    check(host(blocks.eos(Ud, G, dw=dw)), ref, S, torch.float64, "eos")
    ref, S = oracle.v_mag2(D, U, scale=True)
    check(host([blocks.v_mag2(Ud, dw=dw)]), ref, S, torch.float64, "v_mag2")


@pytest.mark.parametrize("dw", [False, True], ids=["f64", "f64dw"])
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("D", [1, 2, 3])
def test_f64_directional_blocks(n, D, dw):
    V, U, W = fields(n, D)
    Ud, _ = quantise(U, torch.float64)
    Wd, _ = quantise(W, torch.float64)
    nv = D + 2
    Gc = synth.cotangent(n, nv)
    Gd, _ = quantise(Gc, torch.float64)
    ref, S = oracle.flux(D, -1, G, U, scale=True)
    check(host(blocks.flux(Ud, -1, G, dw=dw)), ref, S, torch.float64, "flux all")
    for d in range(D):
        ref, S = oracle.flux(D, d, G, U, scale=True)
        check(host(blocks.flux(Ud, d, G, dw=dw)), ref, S, torch.float64, f"flux {d}")
        ref, S = oracle.flux_jac(D, d, G, U, scale=True)
        check(host(blocks.flux_jac(Ud, d, G, dw=dw)), ref, S, torch.float64, f"flux_jac {d}")
        ref, S = oracle.riemann_inv(D, d, G, U, scale=True)
        wm, wp, s = blocks.riemann_inv(Ud, d, G, entropy=True, dw=dw)
        check(host([wm, wp, s]), ref, S, torch.float64, f"riemann {d}")
        for inv in (False, True):
            ref, S = oracle.char_transform(D, d, G, U, W, inverse=inv, scale=True)
            check(host(blocks.char_transform(Ud, Wd, d, G, inverse=inv, dw=dw)), ref, S, torch.float64,
                  f"char {d} inv={inv}")
        ref, S = oracle.flux_vjp(D, d, G, U, Gc, scale=True)
        check(host(blocks.flux_vjp(Ud, Gd, d, G, dw=dw)), ref, S, torch.float64, f"vjp {d}")
        ref, S = oracle.euler_fused(D, d, G, U, W, scale=True)
        Fo, Ao, Yo = blocks.euler_fused(Ud, Wd, d, G, dw=dw)
        check(host([*Fo, *Ao, *Yo]), ref, S, torch.float64, f"fused {d}")


# ---------------------------------------------------------------------------
# reduced-precision storage
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("D", [1, 3])
def test_reduced_precision_blocks(dtype, D):
    n = 4099
    V, U, W = fields(n, D, seed=77)
    Ud, Uq = quantise(U, dtype)
    Vd, Vq = quantise(V, dtype)
    Wd, Wq = quantise(W, dtype)
    ref, S = oracle.prim_from_cons(D, G, Uq, scale=True)
    check(host(blocks.prim_from_cons(Ud, G)), ref, S, dtype, "prim")
    ref, S = oracle.cons_from_prim(D, G, Vq, scale=True)
    check(host(blocks.cons_from_prim(Vd, G)), ref, S, dtype, "cons")
    ref, S = oracle.eos(D, G, Uq, scale=True)
    check(host(blocks.eos(Ud, G)), ref, S, dtype, "eos")
    for d in range(D):
        ref, S = oracle.riemann_inv(D, d, G, Uq, scale=True)
        wm, wp, s = blocks.riemann_inv(Ud, d, G, entropy=True)
        check(host([wm, wp, s]), ref, S, dtype, "riemann")
        ref, S = oracle.euler_fused(D, d, G, Uq, Wq, scale=True)
        Fo, Ao, Yo = blocks.euler_fused(Ud, Wd, d, G)
        check(host([*Fo, *Ao, *Yo]), ref, S, dtype, f"fused {d}")
        for inv in (False, True):
            ref, S = oracle.char_transform(D, d, G, Uq, Wq, inverse=inv, scale=True)
            check(host(blocks.char_transform(Ud, Wd, d, G, inverse=inv)), ref, S, dtype, "char")
        ref, S = oracle.flux_vjp(D, d, G, Uq, Wq, scale=True)
        check(host(blocks.flux_vjp(Ud, Wd, d, G)), ref, S, dtype, "vjp")


# ---------------------------------------------------------------------------
# semantics: in place, skipped outputs, argument errors with real tensors
# ---------------------------------------------------------------------------

def test_in_place_prim_from_cons():
    n, D = 1003, 3
    V, U, W = fields(n, D)
    Ud, _ = quantise(U, torch.float64)
    rho_ptr = Ud[0].data_ptr()
    out = blocks.prim_from_cons(Ud, G, out=Ud)
    assert out[0].data_ptr() == rho_ptr
    ref, S = oracle.prim_from_cons(D, G, U, scale=True)
    check(host(out), ref, S, torch.float64, "in-place prim")


def test_skipped_outputs():
    n, D = 777, 3
    V, U, W = fields(n, D)
    Ud, _ = quantise(U, torch.float64)
    Wd, _ = quantise(W, torch.float64)
    sentinel = torch.full((n,), 12345.0, dtype=torch.float64, device=DEV)
    F = [torch.empty(n, dtype=torch.float64, device=DEV) for _ in range(15)]
    F[3] = None
    A = [sentinel.clone() if k != 6 else torch.empty(n, dtype=torch.float64, device=DEV) for k in range(25)]
    Fo, Ao, Yo = blocks.euler_fused(Ud, None, 0, G, out=(F, [a if k == 6 else None for k, a in enumerate(A)], None))
    ref = oracle.euler_fused(D, 0, G, U, W)
    for k in range(15):
        if k != 3:
            np.testing.assert_allclose(Fo[k].cpu().numpy(), ref[k], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(Ao[6].cpu().numpy(), ref[15 + 6], rtol=1e-12)
    p, c = blocks.eos(Ud, G, want_p=False)
    assert p is None
    np.testing.assert_allclose(c.cpu().numpy(), oracle.eos(D, G, U)[1], rtol=1e-13)


def test_misaligned_plane_is_rejected():
    base = torch.zeros(1001, dtype=torch.float64, device=DEV)
    U = [base[1:].clone() for _ in range(5)]
    U[2] = base[1:]  # 8-byte offset view
    with pytest.raises(capi.FdbbError) as e:
        blocks.flux(U, 0, G)
    assert e.value.status == 3


def test_dw_out_of_range_points_fall_back_to_fp64():
    """Points whose inputs or derived values leave the double-word range
    (tiny or huge magnitudes, tiny nonzero momentum or weights, non-finite
    values) are computed in IEEE double and still match the oracle."""
    n, D = 4103, 3
    V, U, W = fields(n, D, seed=99)
    U = [u.copy() for u in U]
    W = [w.copy() for w in W]
    # scaled states: rho, m, rhoE scaled together keep the state physical
    for i, sc in ((10, 1e-30), (11, 1e30), (12, 1e-9), (513, 1e12), (4100, 2.0 ** -25)):
        for k in range(5):
            U[k][i] *= sc
    U[1][20] = 1e-40            # tiny nonzero momentum
    U[2][21] = -3e-300
    W[3][30] = 1e-200           # tiny characteristic weight
    W[0][31] = 5e25
    ref, S = oracle.euler_fused(D, 0, G, U, W, scale=True)
    Ud, _ = quantise(U, torch.float64)
    Wd, _ = quantise(W, torch.float64)
    for dj in range(D):
        ref, S = oracle.euler_fused(D, dj, G, U, W, scale=True)
        Fo, Ao, Yo = blocks.euler_fused(Ud, Wd, dj, G, dw=True)
        check(host([*Fo, *Ao, *Yo]), ref, S, torch.float64, f"dw fallback fused {dj}")
        Fn, An, Yn = blocks.euler_fused(Ud, Wd, dj, G)
        check(host([*Fn, *An, *Yn]), ref, S, torch.float64, f"native fused {dj}")
    ref, S = oracle.prim_from_cons(D, G, U, scale=True)
    check(host(blocks.prim_from_cons(Ud, G, dw=True)), ref, S, torch.float64, "dw fallback prim")
    # the flux VJP runs two points per thread in packed double-word arithmetic:
    # a pair with one lane out of range (points 12, 513, 4100 above; the tiny
    # and huge cotangents below) or both (10, 11) falls back as a whole, and
    # n = 4103 leaves a one-point tail
    Gc = [g.copy() for g in synth.cotangent(n, 5)]
    Gc[4][41] = 1e-35
    Gc[1][50] = 3e27
    Gd, _ = quantise(Gc, torch.float64)
    for d in range(D):
        ref, S = oracle.flux_vjp(D, d, G, U, Gc, scale=True)
        check(host(blocks.flux_vjp(Ud, Gd, d, G, dw=True)), ref, S, torch.float64, f"dw fallback vjp {d}")
    # a NaN state gives NaN outputs in both arithmetics
    U[0][40] = np.nan
    Ud, _ = quantise(U, torch.float64)
    p_dw, _ = blocks.eos(Ud, G, dw=True)
    p_nat, _ = blocks.eos(Ud, G)
    assert torch.isnan(p_dw[40]) and torch.isnan(p_nat[40])


def test_dw_out_of_range_points_fall_back_on_staged_path():
    """The same out-of-range, tiny, huge and non-finite points, at a size
    where the staged kernel runs: most sit inside shared-memory tiles (where
    the IEEE-double fallback recomputes the chunk from the staged inputs), a
    few in the ragged tail.  Fused pass (every Jacobian direction), packed
    flux VJP (pairs with one or both lanes out of range) and cons -> prim."""
    n, D = staged_n(1024, 4103), 3
    V, U, W = fields(n, D, seed=98)
    U = [u.copy() for u in U]
    W = [w.copy() for w in W]
    last = n - 300  # inside the last 256- and 512-point tiles
    scaled = ((10, 1e-30), (11, 1e30), (12, 1e-9), (513, 1e12), (4100, 2.0 ** -25), (70001, 1e-20),
              (70002, 3e20), (last, 1e-12), (n - 3, 1e15), (n - 1, 2.0 ** -26))
    for i, sc in scaled:
        for k in range(5):
            U[k][i] *= sc
    U[1][20] = 1e-40            # tiny nonzero momentum
    U[2][21] = -3e-300
    U[3][90001] = 1e-38
    W[3][30] = 1e-200           # tiny characteristic weight
    W[0][31] = 5e25
    W[4][n - 2] = 1e-33         # in the tail
    Ud, _ = quantise(U, torch.float64)
    Wd, _ = quantise(W, torch.float64)
    for dj in range(D):
        ref, S = oracle.euler_fused(D, dj, G, U, W, scale=True)
        Fo, Ao, Yo = blocks.euler_fused(Ud, Wd, dj, G, dw=True)
        assert_staged()
        check(host([*Fo, *Ao, *Yo]), ref, S, torch.float64, f"staged dw fallback fused {dj}")
    ref, S = oracle.prim_from_cons(D, G, U, scale=True)
    Vo = blocks.prim_from_cons(Ud, G, dw=True)
    assert_staged()
    check(host(Vo), ref, S, torch.float64, "staged dw fallback prim")
    Gc = [g.copy() for g in synth.cotangent(n, 5)]
    Gc[4][41] = 1e-35
    Gc[1][50] = 3e27
    Gc[2][last + 1] = 1e-30
    Gd, _ = quantise(Gc, torch.float64)
    for d in range(D):
        ref, S = oracle.flux_vjp(D, d, G, U, Gc, scale=True)
        gU = blocks.flux_vjp(Ud, Gd, d, G, dw=True)
        assert_staged()
        check(host(gU), ref, S, torch.float64, f"staged dw fallback vjp {d}")
    # a NaN state inside a staged tile gives NaN in both arithmetics
    U[0][4000] = np.nan
    Ud, _ = quantise(U, torch.float64)
    p_dw, _ = blocks.eos(Ud, G, dw=True)
    assert_staged()
    p_nat, _ = blocks.eos(Ud, G)
    assert torch.isnan(p_dw[4000]) and torch.isnan(p_nat[4000])
    assert capi.device_status() == 0


def test_dw_copies_are_bit_exact():
    n, D = 1001, 3
    V, U, W = fields(n, D, seed=5)
    Ud, _ = quantise(U, torch.float64)
    Wd, _ = quantise(W, torch.float64)
    F, A, Y = blocks.euler_fused(Ud, Wd, 0, G, dw=True)
    for d in range(D):
        assert torch.equal(F[d * 5], Ud[1 + d])
    Vo = blocks.prim_from_cons(Ud, G, dw=True)
    assert torch.equal(Vo[0], Ud[0])


def test_dw_rebuild_across_a_power_of_two():
    """A double-word result hi + lo whose hi is a power of two and whose lo
    has the opposite sign lies in the binade below hi, where a double's unit
    in the last place is half as large; the rebuilt double must still be
    hi + lo.  Primitive-form flux at rho = u = 1, p = 1 - 2^-26:
    F_x[1] = rho u^2 + p = 2 - 2^-26 (hi = 2, lo = -2^-26); at rho = 2,
    u = 1, v = -(1 - 2^-27): F_x[2] = rho u v = -2 + 2^-26 (hi = -2,
    lo = 2^-26).  Both are doubles and come out of the double-word arithmetic
    without rounding, so the result is exact to far below the 2^-27 that a
    rebuild in the wrong binade would be off by.  The fused pass on the
    conservative form of the first state, at a size where the staged kernel
    runs, takes the same step against the oracle."""
    n = 4099
    V = [np.ones(n), np.ones(n), np.zeros(n), np.zeros(n), np.full(n, 1 - 2.0 ** -26)]
    V[0][1::2] = 2.0
    V[2][1::2] = -(1 - 2.0 ** -27)
    V[4][1::2] = 1.0
    Vd, _ = quantise(V, torch.float64)
    for dw in (True, False):
        F = host(blocks.flux_prim(Vd, 0, G, dw=dw))
        assert np.all(np.abs(F[1][0::2] - (2 - 2.0 ** -26)) <= 2.0 ** -40), dw
        assert np.all(np.abs(F[2][1::2] - (-2 + 2.0 ** -26)) <= 2.0 ** -40), dw
    m = staged_n(512, 7)
    U1 = oracle.cons_from_prim(3, G, [np.array([v[0]]) for v in V])
    U = [np.full(m, u[0]) for u in U1]
    W = synth.char_weights(m, 5, seed=3)
    Ud, _ = quantise(U, torch.float64)
    Wd, _ = quantise(W, torch.float64)
    F, A, Y = blocks.euler_fused(Ud, Wd, 0, G, dw=True)
    assert_staged()
    ref, S = oracle.euler_fused(3, 0, G, U, W, scale=True)
    got = host([*F, *A, *Y])
    assert abs(ref[1][0] - 2.0) < 2.0 ** -24 and ref[1][0] < 2.0  # the case this test is about
    check(got, ref, S, torch.float64, "fused at a power of two")


# ---------------------------------------------------------------------------
# full size, in the benchmark's launch configuration
# ---------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("dtype,dw", [(torch.float64, False), (torch.float64, True), (torch.float32, False),
                                      (torch.bfloat16, False)],
                         ids=["f64", "f64dw", "f32", "bf16"])
def test_full_size_fused_sampled(dtype, dw):
    """3D fused pass at N = 2^26 (the benchmark size): sampled points against
    the oracle, and A_x(U) U = F_x(U) checked at every point."""
    n, D = 1 << 26, 3
    V = synth.euler3d(n)
    U = oracle.cons_from_prim(D, G, V)
    W = synth.char_weights(n)
    Ud, Uq = quantise(U, dtype)
    Wd, Wq = quantise(W, dtype)
    del V
    F, A, Y = blocks.euler_fused(Ud, Wd, 0, G, dw=dw)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.integers(0, n, 4096), np.arange(n - 37, n), np.arange(5)]))
    it = torch.from_numpy(idx).to(DEV)
    got = [t[it].double().cpu().numpy() for t in (*F, *A, *Y)]
    Us = [u[idx] for u in Uq]
    Ws = [w[idx] for w in Wq]
    ref, S = oracle.euler_fused(D, 0, G, Us, Ws, scale=True)
    check(got, ref, S, dtype, "full-size fused")
    # homogeneity at every point, evaluated on the device in float64 (each
    # output rounded to the storage type once: 2 u_store of the scale more;
    # points whose stored state is below vacuum give NaN on both sides)
    Ux = [u.double() for u in Ud]
    tol = 1e-12 if dtype == torch.float64 else 64 * 2.0 ** -24
    for r in range(5):
        Au = sum(A[r * 5 + c].double() * Ux[c] for c in range(5))
        scale = sum((A[r * 5 + c].double() * Ux[c]).abs() for c in range(5))
        err = (Au - F[r].double()).abs()
        ok = err <= (8 * tol + 2 * U_STORE[dtype]) * (scale + F[r].double().abs()) + 1e-300
        if dtype == torch.bfloat16:
            ok = ok | torch.isnan(err)
        assert bool(ok.all()), r


# ---------------------------------------------------------------------------
# the shared-memory-staged kernels (taken once every SM has >= 4 tiles)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,dw", [(torch.float64, False), (torch.float64, True), (torch.float32, False),
                                      (torch.bfloat16, False), (torch.float16, False)],
                         ids=["f64", "f64dw", "f32", "bf16", "f16"])
def test_staged_path_parity(dtype, dw):
    """n = 4 tiles per SM of the widest tile (1024 points) plus a ragged tail,
    every point against the oracle, for ops with 5, 10 and 10-with-skipped-W
    input planes; each call is checked to have taken the staged kernel."""
    n = staged_n(1024, 4099)
    D = 3
    V, U, W = fields(n, D, seed=2024)
    Ud, Uq = quantise(U, dtype)
    Wd, Wq = quantise(W, dtype)
    Gc = synth.cotangent(n, 5)
    Gd, Gq = quantise(Gc, dtype)
    ref, S = oracle.euler_fused(D, 1, G, Uq, Wq, scale=True)
    Fo, Ao, Yo = blocks.euler_fused(Ud, Wd, 1, G, dw=dw)
    assert_staged()
    check(host([*Fo, *Ao, *Yo]), ref, S, dtype, "staged fused")
    Fo, Ao, _ = blocks.euler_fused(Ud, None, 2, G, out=(blocks._alloc(15, n, dtype, DEV),
                                                        blocks._alloc(25, n, dtype, DEV), None), dw=dw)
    assert_staged()
    ref, S = oracle.euler_fused(D, 2, G, Uq, Wq, scale=True)
    check(host([*Fo, *Ao]), ref[:40], S[:40], dtype, "staged fused without W")
    ref, S = oracle.flux_vjp(D, 0, G, Uq, Gq, scale=True)
    gU = blocks.flux_vjp(Ud, Gd, 0, G, dw=dw)
    assert_staged()
    check(host(gU), ref, S, dtype, "staged vjp")
    ref, S = oracle.prim_from_cons(D, G, Uq, scale=True)
    Vo = blocks.prim_from_cons(Ud, G, dw=dw)
    assert_staged()
    check(host(Vo), ref, S, dtype, "staged prim")
    ref, S = oracle.v_mag2(D, Uq, scale=True)
    y = blocks.v_mag2(Ud, dw=dw)
    assert_staged()
    check(host([y]), ref, S, dtype, "staged v_mag2")
    assert capi.device_status() == 0  # no bounded wait ran out


def test_staged_fused_with_skipped_flux_planes():
    """The staged double-word fused pass (two points per thread, packed) with
    NULL flux and Jacobian planes: every other plane is still correct."""
    n, D = staged_n(512, 77), 3
    V, U, W = fields(n, D, seed=515)
    Ud, _ = quantise(U, torch.float64)
    Wd, _ = quantise(W, torch.float64)
    F = blocks._alloc(15, n, torch.float64, DEV)
    A = blocks._alloc(25, n, torch.float64, DEV)
    Y = blocks._alloc(5, n, torch.float64, DEV)
    Fo = [None if k in (0, 3, 7, 14) else f for k, f in enumerate(F)]
    Ao = [None if k in (1, 24) else x for k, x in enumerate(A)]
    blocks.euler_fused(Ud, Wd, 2, G, out=(Fo, Ao, Y), dw=True)
    assert_staged()
    ref, S = oracle.euler_fused(D, 2, G, U, W, scale=True)
    keep = [k for k in range(15) if Fo[k] is not None] + [15 + k for k in range(25) if Ao[k] is not None] + \
        list(range(40, 45))
    got = host([*F, *A, *Y])
    check([got[k] for k in keep], [ref[k] for k in keep], [S[k] for k in keep], torch.float64, "staged fused, skips")


def _floored_field(n, seed):
    """A 3D field (and weights) whose momenta and weights all have magnitude
    >= 1e-5, so no point leaves the double-word range and falls back."""
    _, U, W = fields(n, 3, seed=seed)
    floor = lambda x: np.where(np.abs(x) < 1e-5, np.copysign(1e-5, x), x)
    return [U[0], *(floor(m) for m in U[1:4]), U[4]], [floor(w) for w in W]


@pytest.mark.parametrize("staged", [False, True], ids=["direct", "staged"])
def test_packed_blocks_lanes_are_independent(staged):
    """Every double-word block that runs two points per thread as the lanes
    of packed FP32x2 values gives a point the same bits whatever point shares
    its pair: the field shifted by one point re-pairs every point."""
    n = staged_n(1024, 1001) if staged else 4099
    U, W = _floored_field(n + 1, 78)
    Ud = [torch.from_numpy(u).to(DEV) for u in U]
    Wd = [torch.from_numpy(w).to(DEV) for w in W]
    first = lambda ts: [t[:n].clone() for t in ts]
    second = lambda ts: [t[1:].clone() for t in ts]
    calls = {
        "fused": lambda U_, W_: [*sum(blocks.euler_fused(U_, W_, 1, G, dw=True), [])],
        "v_mag2": lambda U_, W_: [blocks.v_mag2(U_, dw=True)],
        "eos": lambda U_, W_: list(blocks.eos(U_, G, dw=True)),
        "prim": lambda U_, W_: blocks.prim_from_cons(U_, G, dw=True),
        "riemann": lambda U_, W_: list(blocks.riemann_inv(U_, 2, G, dw=True)[:2]),
        "flux_all": lambda U_, W_: blocks.flux(U_, -1, G, dw=True),
        "jac": lambda U_, W_: blocks.flux_jac(U_, 0, G, dw=True),
        "char_fwd": lambda U_, W_: blocks.char_transform(U_, W_, 1, G, dw=True),
        "char_inv": lambda U_, W_: blocks.char_transform(U_, W_, 2, G, inverse=True, dw=True),
        "temperature": lambda U_, W_: [blocks.temperature(U_, 2.5, G, dw=True)],
        "vjp": lambda U_, W_: blocks.flux_vjp(U_, W_, 2, G, dw=True),
    }
    for name, fn in calls.items():
        a = fn(first(Ud), first(Wd))
        kind = capi.last_launch()
        assert kind.points_per_thread == 2, name
        assert kind.kernel == (capi.FDBB_KERNEL_STAGED if staged else capi.FDBB_KERNEL_DIRECT), name
        b = fn(second(Ud), second(Wd))
        for k, (x, y) in enumerate(zip(a, b)):
            assert torch.equal(x[1:], y[:-1]), (name, k)
    V = [torch.from_numpy(v).to(DEV) for v in oracle.prim_from_cons(3, G, U)]
    for name, fn in {"flux_prim": lambda V_: blocks.flux_prim(V_, -1, G, dw=True),
                     "jac_prim": lambda V_: blocks.flux_jac_prim(V_, 1, G, dw=True)}.items():
        a, b = fn(first(V)), fn(second(V))
        assert capi.last_launch().points_per_thread == 2, name
        for k, (x, y) in enumerate(zip(a, b)):
            assert torch.equal(x[1:], y[:-1]), (name, k)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("staged", [False, True], ids=["direct", "staged"])
def test_packed_float_lanes_are_independent(staged, dtype):
    """The float-arithmetic blocks evaluate a thread's four points as two
    packed FP32x2 pairs: a point's bits do not depend on which point shares
    its pair or its thread (the field shifted by one point re-pairs them).
    Bit patterns are compared, so NaNs of states that are non-physical once
    rounded to 16 bits compare equal too."""
    ibits = {torch.float32: torch.int32, torch.bfloat16: torch.int16}[dtype]
    same = lambda x, y: torch.equal(x.view(ibits), y.view(ibits))
    n = staged_n(1024, 1001) if staged else 4099
    _, U, W = fields(n + 1, 3, seed=79)
    Ud = [torch.from_numpy(u).to(DEV).to(dtype) for u in U]
    Wd = [torch.from_numpy(w).to(DEV).to(dtype) for w in W]
    first = lambda ts: [t[:n].clone() for t in ts]
    second = lambda ts: [t[1:].clone() for t in ts]
    calls = {
        "eos": lambda U_, W_: list(blocks.eos(U_, G)),
        "riemann": lambda U_, W_: list(blocks.riemann_inv(U_, 2, G, entropy=True)),
        "char_fwd": lambda U_, W_: blocks.char_transform(U_, W_, 0, G),
        "flux_all": lambda U_, W_: blocks.flux(U_, -1, G),
        "jac": lambda U_, W_: blocks.flux_jac(U_, 1, G),
        "vjp": lambda U_, W_: blocks.flux_vjp(U_, W_, 2, G),
        "roe": lambda U_, W_: blocks.roe_flux(U_, [torch.roll(u, 1) for u in U_], 1, G),
        "temperature": lambda U_, W_: [blocks.temperature(U_, 2.5, G)],
    }
    for name, fn in calls.items():
        a = fn(first(Ud), first(Wd))
        assert capi.last_launch().kernel == (capi.FDBB_KERNEL_STAGED if staged else capi.FDBB_KERNEL_DIRECT), name
        b = fn(second(Ud), second(Wd))
        for k, (x, y) in enumerate(zip(a, b)):
            if name == "roe":
                # U_R is the field rolled by one point: point j of the first
                # call and point j - 1 of the second see the same (U_L, U_R)
                # for j >= 2 (away from the roll's seam)
                assert same(x[2:], y[1:-1]), (name, k)
            else:
                assert same(x[1:], y[:-1]), (name, k)


@pytest.mark.parametrize("staged", [False, True], ids=["direct", "staged"])
def test_packed_vjp_lanes_are_independent(staged):
    """The double-word flux VJP runs two points per thread as the two lanes of
    packed FP32x2 values.  A point's result must not depend on the point that
    shares its pair: shifting the field by one point re-pairs every point, and
    the results are the same bits (in-range fields, so no pair falls back)."""
    D = 3
    n = staged_n(512, 1001) if staged else 4099
    _, U, _ = fields(n + 1, D, seed=77)
    Gc = synth.cotangent(n + 1, 5)
    # keep every momentum and cotangent at magnitude >= 1e-5 (a normal draw
    # below 2^-24 would send its pair to the IEEE fallback)
    floor = lambda x: np.where(np.abs(x) < 1e-5, np.copysign(1e-5, x), x)
    U = [U[0], *(floor(m) for m in U[1:4]), U[4]]
    Gc = [floor(g) for g in Gc]
    Ud = [torch.from_numpy(u).to(DEV) for u in U]
    Gd = [torch.from_numpy(g).to(DEV) for g in Gc]
    a = blocks.flux_vjp([u[:n].clone() for u in Ud], [g[:n].clone() for g in Gd], 0, G, dw=True)
    b = blocks.flux_vjp([u[1:].clone() for u in Ud], [g[1:].clone() for g in Gd], 0, G, dw=True)
    kind = capi.last_launch().kernel
    assert kind == (capi.FDBB_KERNEL_STAGED if staged else capi.FDBB_KERNEL_DIRECT)
    for k in range(5):
        assert torch.equal(a[k][1:], b[k][:-1]), k


def test_fused_over_host_buffers_matches_device_call():
    """blocks.euler_fused_host (pinned host fields, chunked pipeline) gives the
    same bits as the device-resident call."""
    n, D = 3 * (1 << 18) + 5, 3
    V, U, W = fields(n, D, seed=31)
    hU = [torch.from_numpy(u).pin_memory() for u in U]
    hW = [torch.from_numpy(w).pin_memory() for w in W]
    out = tuple([torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(k)] for k in (15, 25, 5))
    work = blocks.euler_fused_host(hU, hW, out, 0, G, chunk=(1 << 18) + 6)
    work = blocks.euler_fused_host(hU, hW, out, 0, G, chunk=(1 << 18) + 6, work=work)
    torch.cuda.synchronize()
    Fd, Ad, Yd = blocks.euler_fused([u.to(DEV) for u in hU], [w.to(DEV) for w in hW], 0, G)
    for h, d in zip([*out[0], *out[1], *out[2]], [*Fd, *Ad, *Yd]):
        assert torch.equal(h, d.cpu())


# ---------------------------------------------------------------------------
# Roe flux and Roe-averaged characteristic transform
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,dw", [(torch.float64, False), (torch.float64, True), (torch.float32, False),
                                      (torch.bfloat16, False)], ids=["f64", "f64dw", "f32", "bf16"])
@pytest.mark.parametrize("n", [7, 4099])
@pytest.mark.parametrize("D", [1, 2, 3])
def test_roe_blocks(D, n, dtype, dw):
    _, UL, W = fields(n, D, seed=300)
    _, UR, _ = fields(n, D, seed=301)
    ULd, ULq = quantise(UL, dtype)
    URd, URq = quantise(UR, dtype)
    Wd, Wq = quantise(W, dtype)
    for d in range(D):
        ref, S = oracle.roe_flux(D, d, G, ULq, URq, scale=True)
        check(host(blocks.roe_flux(ULd, URd, d, G, dw=dw)), ref, S, dtype, f"roe flux {d}")
        for inv in (False, True):
            ref, S = oracle.roe_char_transform(D, d, G, ULq, URq, Wq, inverse=inv, scale=True)
            check(host(blocks.roe_char_transform(ULd, URd, Wd, d, G, inverse=inv, dw=dw)), ref, S, dtype,
                  f"roe char {d} inv={inv}")


@pytest.mark.parametrize("dw", [False, True], ids=["f64", "f64dw"])
def test_roe_flux_staged_path(dw):
    n, D = staged_n(512, 333), 3
    _, UL, _ = fields(n, D, seed=310)
    _, UR, _ = fields(n, D, seed=311)
    ULd, _ = quantise(UL, torch.float64)
    URd, _ = quantise(UR, torch.float64)
    ref, S = oracle.roe_flux(D, 1, G, UL, UR, scale=True)
    F = blocks.roe_flux(ULd, URd, 1, G, dw=dw)
    assert_staged()
    check(host(F), ref, S, torch.float64, "staged roe flux")


# ---------------------------------------------------------------------------
# primitive-variable forms and temperature
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,dw", [(torch.float64, False), (torch.float64, True), (torch.float32, False),
                                      (torch.bfloat16, False)], ids=["f64", "f64dw", "f32", "bf16"])
@pytest.mark.parametrize("n", [7, 4099])
@pytest.mark.parametrize("D", [1, 2, 3])
def test_primitive_forms_and_temperature(D, n, dtype, dw):
    V, U, _ = fields(n, D, seed=400)
    Vd, Vq = quantise(V, dtype)
    Ud, Uq = quantise(U, dtype)
    ref, S = oracle.flux_prim(D, -1, G, Vq, scale=True)
    check(host(blocks.flux_prim(Vd, -1, G, dw=dw)), ref, S, dtype, "flux_prim all")
    for d in range(D):
        ref, S = oracle.flux_prim(D, d, G, Vq, scale=True)
        check(host(blocks.flux_prim(Vd, d, G, dw=dw)), ref, S, dtype, f"flux_prim {d}")
        ref, S = oracle.flux_jac_prim(D, d, G, Vq, scale=True)
        check(host(blocks.flux_jac_prim(Vd, d, G, dw=dw)), ref, S, dtype, f"flux_jac_prim {d}")
    for cv in (2.5, 0.7):
        ref, S = oracle.temperature(D, G, cv, Uq, scale=True)
        check(host([blocks.temperature(Ud, cv, G, dw=dw)]), ref, S, dtype, f"temperature cv={cv}")
