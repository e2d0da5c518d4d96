"""Batched Rusanov finite-volume steps and the serving loop on the GPU.

FP64 grids match the FP64 oracle (same scheme, different operation order)
to 1e-11 of the field's magnitude after several steps, with the same time
steps; FP32 grids match it to 2e-5.  A grid's results are bitwise the same
whether it runs alone or batched with other grids, and a served request's
answer is bitwise the same alone and in the mix.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_09851_gb300 import fv, serve, synth

pytestmark = pytest.mark.gpu
G_ = 1.4
DEV = "cuda:0"


def _initial(n, seed, swirl=0.3):
    V = synth.smooth_perturbation(n, seed)
    x = (np.arange(n) + 0.5) / n
    V[1] = V[1] + swirl * np.broadcast_to(np.sin(2 * np.pi * x)[None, :, None], (n, n, n)).reshape(-1)
    V[3] = V[3] - 0.5 * swirl * np.broadcast_to(np.cos(2 * np.pi * x)[None, None, :], (n, n, n)).reshape(-1)
    return oracle.cons_from_prim(3, G_, V)


def _dev(U, dtype):
    return [torch.from_numpy(u).to(DEV).to(dtype) for u in U]


@pytest.mark.parametrize("n,steps", [(8, 5), (13, 4)])
def test_fv_fp64_matches_oracle(n, steps):
    U = _initial(n, 3)
    smax = torch.zeros(3 * 4, dtype=torch.float64, device=DEV)
    g = fv.grid_from_conservative(_dev(U, torch.float64), n, 1, smax, G_, dt_log_steps=steps)
    for _ in range(steps):
        fv.rusanov_step([g], smax, G_, 0.4)
    torch.cuda.synchronize()
    ref, dts = oracle.rusanov_run(n, G_, 0.4, steps, U)
    np.testing.assert_allclose(g.dt_log.cpu().numpy(), dts, rtol=1e-13)
    for k in range(5):
        got = g.U[k].cpu().numpy()
        assert np.abs(got - ref[k]).max() <= 1e-11 * max(1.0, np.abs(ref[k]).max()), k


def test_fv_fp32_matches_oracle():
    n, steps = 12, 10
    U = _initial(n, 4)
    Uq = [u.astype(np.float32).astype(np.float64) for u in U]
    smax = torch.zeros(3, dtype=torch.float32, device=DEV)
    g = fv.grid_from_conservative(_dev(Uq, torch.float32), n, 0, smax, G_, dt_log_steps=steps)
    for _ in range(steps):
        fv.rusanov_step([g], smax, G_, 0.4)
    ref, dts = oracle.rusanov_run(n, G_, 0.4, steps, Uq)
    np.testing.assert_allclose(g.dt_log.cpu().numpy(), dts, rtol=1e-5)
    for k in range(5):
        got = g.U[k].double().cpu().numpy()
        assert np.abs(got - ref[k]).max() <= 2e-5 * max(1.0, np.abs(ref[k]).max()), k
    # conservation of mass, momentum and energy (to float roundoff)
    for k in range(5):
        tot0, tot = Uq[k].sum(), g.U[k].double().sum().item()
        assert abs(tot - tot0) <= 1e-5 * max(1.0, np.abs(Uq[k]).sum())


@pytest.mark.parametrize("n", [33, 45, 64])
def test_fv_fp32_across_plane_segments(n):
    """FP32 grids taller than one column segment (a lone small grid is cut
    into 16-plane segments): the z face between two segments is formed by
    both tiles (as the upper face of the lower tile's last plane pair and as
    the carried lower face of the upper tile), and a segment of odd length
    ends with a half-used plane pair (33 = 2 x 16 + 1, 45 = 2 x 16 + 13).
    Matches the FP64 oracle to 2e-5 and conserves mass, momentum and energy
    to float rounding."""
    steps = 3
    U = _initial(n, 6)
    Uq = [u.astype(np.float32).astype(np.float64) for u in U]
    smax = torch.zeros(3, dtype=torch.float32, device=DEV)
    g = fv.grid_from_conservative(_dev(Uq, torch.float32), n, 0, smax, G_, dt_log_steps=steps)
    for _ in range(steps):
        fv.rusanov_step([g], smax, G_, 0.4)
    ref, dts = oracle.rusanov_run(n, G_, 0.4, steps, Uq)
    np.testing.assert_allclose(g.dt_log.cpu().numpy(), dts, rtol=1e-5)
    for k in range(5):
        got = g.U[k].double().cpu().numpy()
        assert np.abs(got - ref[k]).max() <= 2e-5 * max(1.0, np.abs(ref[k]).max()), (n, k)
        tot0, tot = Uq[k].sum(), got.sum()
        assert abs(tot - tot0) <= 1e-5 * max(1.0, np.abs(Uq[k]).sum()), (n, k)


@pytest.mark.parametrize("n", [12, 45])
def test_fv_fp32_plane_pairing_is_invisible(n):
    """FP32 grids run two z planes per thread as the lanes of packed FP32x2
    values, in column segments of an even number of planes.  Rolling the periodic grid by one
    plane in z re-pairs every plane and moves every segment boundary relative
    to the data, and the result is the rolled result bit for bit: a face is the
    same packed sequence in either lane, and a carried lower face the same as
    the upper face the tile below forms."""
    steps = 3
    U = [u.astype(np.float32) for u in _initial(n, 8)]
    roll = lambda u: np.roll(u.reshape(n, n, n), 1, axis=0).reshape(-1)
    outs = []
    for V in (U, [roll(u) for u in U]):
        smax = torch.zeros(3, dtype=torch.float32, device=DEV)
        g = fv.grid_from_conservative([torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for v in V], n, 0, smax, G_)
        for _ in range(steps):
            fv.rusanov_step([g], smax, G_, 0.4)
        outs.append([t.cpu().numpy() for t in g.U])
    for k in range(5):
        assert np.array_equal(roll(outs[0][k]), outs[1][k]), k


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_fv_batched_equals_alone(dtype):
    sizes = [3, 5, 8, 13, 16, 7]
    steps = 6
    Us = [_initial(n, 10 + i) for i, n in enumerate(sizes)]
    smax_a = torch.zeros(3 * len(sizes), dtype=dtype, device=DEV)
    alone = []
    for i, (n, U) in enumerate(zip(sizes, Us)):
        g = fv.grid_from_conservative(_dev(U, dtype), n, i, smax_a, G_)
        for _ in range(steps):
            fv.rusanov_step([g], smax_a, G_, 0.4)
        alone.append(g)
    smax_b = torch.zeros(3 * len(sizes), dtype=dtype, device=DEV)
    together = [fv.grid_from_conservative(_dev(U, dtype), n, len(sizes) - 1 - i, smax_b, G_)
                for i, (n, U) in enumerate(zip(sizes, Us))]
    # staggered: the first half starts two steps earlier
    for _ in range(2):
        fv.rusanov_step(together[:3], smax_b, G_, 0.4)
    for s in range(steps - 2):
        fv.rusanov_step(together, smax_b, G_, 0.4)
    for _ in range(2):
        fv.rusanov_step(together[3:], smax_b, G_, 0.4)
    for a, b in zip(alone, together):
        assert a.step == b.step == steps
        for k in range(5):
            assert torch.equal(a.U[k], b.U[k])


def test_fv_many_grids_over_one_table():
    """More grids than one descriptor table holds (two launches per step)."""
    sizes = [2 + (i % 5) for i in range(300)]
    smax = torch.zeros(3 * 300, dtype=torch.float32, device=DEV)
    grids = [fv.grid_from_conservative(_dev(_initial(n, 100 + i), torch.float32), n, i, smax, G_)
             for i, n in enumerate(sizes)]
    for _ in range(3):
        fv.rusanov_step(grids, smax, G_, 0.4)
    g = grids[257]
    ref, _ = oracle.rusanov_run(g.n, G_, 0.4, 3,
                                [u.astype(np.float32).astype(np.float64) for u in _initial(g.n, 100 + 257)])
    for k in range(5):
        assert np.abs(g.U[k].double().cpu().numpy() - ref[k]).max() <= 2e-5 * max(1.0, np.abs(ref[k]).max())


def test_serving_alone_equals_mixed():
    reqs = synth.request_stream(12, rate=2e5, n_lo=6, n_hi=24, steps_lo=5, steps_hi=15, seed=77)
    srv = serve.FVServer(DEV, torch.float32, keep_results=True)
    rep = srv.run(reqs, realtime=True)
    assert sorted(rep.latencies) == [r.rid for r in reqs]
    assert rep.max_active > 1  # requests really overlapped
    for r in reqs[:5]:
        one = serve.FVServer(DEV, torch.float32, keep_results=True).run([r], realtime=False)
        for k in range(5):
            assert torch.equal(one.results[r.rid][k], rep.results[r.rid][k]), (r.rid, k)
    s = rep.summary()
    assert s["p99_s"] >= s["p50_s"] > 0


def test_serving_admission_by_budget():
    reqs = synth.request_stream(6, rate=1e6, n_lo=10, n_hi=10, steps_lo=3, steps_hi=3, seed=5)
    big = synth.Request(rid=99, arrival=0.0, n=64, steps=2, seed=1)
    one_grid = 2 * 5 * 10 ** 3 * 4
    srv = serve.FVServer(DEV, torch.float32, hbm_budget=one_grid + 100)
    rep = srv.run(reqs + [big], realtime=False)
    assert rep.max_active == 1
    assert rep.rejected == [99]
    assert len(rep.latencies) == 6


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 3e-6)], ids=["f64", "f32"])
@pytest.mark.parametrize("n", [1, 7, 32, 50])
def test_smooth_initial_state_on_device(n, dtype, tol):
    """fdbb_fv_init_smooth builds the serving requests' initial state: it equals
    the host generator's primitive planes converted by the oracle (tolerance:
    a few ulp of the storage type), and its initial wave speed equals the
    oracle's maximum."""
    seed = 11 + n
    smax = torch.zeros(3 * 8, dtype=dtype, device=DEV)
    g = fv.new_grid_smooth(n, seed, 2, smax, dtype, DEV, G_)
    torch.cuda.synchronize()
    ref = oracle.cons_from_prim(3, G_, synth.smooth_perturbation(n, seed))
    for k in range(5):
        got = g.U[k].double().cpu().numpy()
        assert np.all(np.abs(got - ref[k]) <= tol * np.maximum(1.0, np.abs(ref[k]))), k
    dt = oracle.rusanov_dt(n, G_, 0.4, ref)
    ref_speed = 0.4 * (1.0 / n) / dt
    assert abs(float(smax[6]) - ref_speed) <= 1e-5 * ref_speed
    # the served request's answer: default initial state equals the host-built one
    reqs = [synth.Request(0, 0.0, 9, 3, 5)]
    a = serve.FVServer(DEV, torch.float64, keep_results=True).run(reqs, realtime=False).results[0]
    b = serve.FVServer(DEV, torch.float64, keep_results=True,
                       initial_state=lambda r: [torch.from_numpy(v).to(DEV) for v in
                                                synth.smooth_perturbation(r.n, r.seed)]).run(reqs, realtime=False).results[0]
    for x, y in zip(a, b):
        assert torch.allclose(x, y, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("axis", [0, 1, 2], ids=["x", "y", "z"])
def test_fv_step_hand_values(axis, dtype):
    """One step of the batched kernels on the 4-cell contact of
    tests/golden/rusanov_contact_step.txt gives the hand-derived density,
    momentum u rho' and energy 2.5 + u^2 rho'/2, and the hand-derived dt, in
    every direction (FP64: 1e-13 relative; FP32: 2e-5)."""
    from test_oracle_pins import _rusanov_golden, contact_state
    n = 4
    tol = 1e-13 if dtype == torch.float64 else 2e-5
    for name, cs in _rusanov_golden().items():
        u = cs["u"]
        U, coord = contact_state(n, axis, u)
        smax = torch.zeros(3, dtype=dtype, device=DEV)
        g = fv.grid_from_conservative(_dev(U, dtype), n, 0, smax, G_, dt_log_steps=1)
        fv.rusanov_step([g], smax, G_, 0.4)
        torch.cuda.synchronize()
        want = np.array([cs["rho"][i] for i in range(n)])[coord]
        np.testing.assert_allclose(g.dt_log.cpu().numpy()[0], cs["dt"], rtol=tol, err_msg=name)
        np.testing.assert_allclose(g.U[0].double().cpu().numpy(), want, rtol=tol, err_msg=name)
        np.testing.assert_allclose(g.U[1 + axis].double().cpu().numpy(), u * want, rtol=tol, atol=tol,
                                   err_msg=name)
        np.testing.assert_allclose(g.U[4].double().cpu().numpy(), 2.5 + 0.5 * u * u * want, rtol=tol,
                                   err_msg=name)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_serving_stops_and_resumes_bit_for_bit(dtype):
    """A run stopped after a few batched steps copies its unfinished requests'
    state to host memory; a fresh server resumes them from those snapshots
    (and starts the ones never admitted).  Every request's final state equals
    the uninterrupted run's bit for bit: the resumed time step comes from the
    same exact maximum of the same state."""
    shapes = [(16, 9), (23, 14), (18, 5), (31, 12), (20, 20), (17, 7), (25, 3)]
    reqs = [synth.Request(i, 0.0, n, st, 500 + i) for i, (n, st) in enumerate(shapes)]
    full = serve.FVServer(DEV, dtype, keep_results=True).run(reqs, realtime=False)
    part = serve.FVServer(DEV, dtype, keep_results=True, max_active=4).run(reqs, realtime=False, max_iterations=6)
    assert part.snapshots, "the stopped run left no request unfinished"
    for rid, snap in part.snapshots.items():
        assert 0 < snap.step < reqs[rid].steps and snap.U[0].device.type == "cpu"
    rest_ids = set(part.snapshots) | set(part.unstarted)
    assert not rest_ids & set(part.results)
    rest = serve.FVServer(DEV, dtype, keep_results=True).run([r for r in reqs if r.rid in rest_ids],
                                                             realtime=False, resume=part.snapshots)
    results = {**part.results, **rest.results}
    assert set(results) == {r.rid for r in reqs}
    for rid, U in full.results.items():
        for k, (a, b) in enumerate(zip(U, results[rid])):
            assert torch.equal(a, b), (rid, k)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_fv_segment_length_is_invisible(dtype):
    """The step kernel cuts columns into segments whose length (64, 32 or 16
    planes) depends on how many tiles a launch has.  A grid stepped alone
    (few tiles: short segments) and in a batch with eight 128^3 grids (many
    tiles: long segments) ends with the same bits."""
    n, steps = 75, 3
    U = _dev(_initial(n, 9), dtype)
    smax = torch.zeros(3 * 9, dtype=dtype, device=DEV)
    alone = fv.grid_from_conservative(U, n, 0, smax, G_)
    for _ in range(steps):
        fv.rusanov_step([alone], smax, G_, 0.4)
    fillers = [fv.new_grid_smooth(128, 90 + i, 1 + i, smax, dtype, DEV) for i in range(8)]
    mixed = fv.grid_from_conservative(U, n, 0, smax, G_)
    for _ in range(steps):
        fv.rusanov_step([*fillers[:4], mixed, *fillers[4:]], smax, G_, 0.4)
    torch.cuda.synchronize()
    for k in range(5):
        assert torch.equal(alone.U[k], mixed.U[k]), k
