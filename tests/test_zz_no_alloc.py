"""The allocation-free finite-volume step, fdbb_fv_rusanov_step_noalloc.

Some callers cannot allocate device memory: their host framework owns all of
it, or their loop must not synchronise the device.  This entry point keeps the
per-grid wave-speed scratch in a fixed array of the library's own device
memory instead of a caller-provided buffer.  Here it is called through the C
ABI twice in a row and compared with the scratch-using path
(fdbb_fv_max_speed + fdbb_fv_rusanov_step): it runs the same kernels on the
same values, so the states and time steps must be identical bit for bit.
They are also checked against the FP64 oracle, within the tolerances of the
other finite-volume tests, and a call after a warm-up call must leave the
device's free memory unchanged.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_09851_gb300 import build, capi, fv, synth

pytestmark = pytest.mark.gpu
G_ = 1.4
CFL = 0.4
DEV = "cuda:0"
TOL = {torch.float32: 2e-5, torch.float64: 1e-11}


def _initial(n, seed):
    V = synth.smooth_perturbation(n, seed)
    x = (np.arange(n) + 0.5) / n
    V[1] = V[1] + 0.3 * np.broadcast_to(np.sin(2 * np.pi * x)[None, :, None], (n, n, n)).reshape(-1)
    return oracle.cons_from_prim(3, G_, V)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_noalloc_step_matches_scratch_step(dtype):
    build.build()
    sizes = [5, 12, 9, 1]
    steps = 2
    code = capi.FDBB_F32 if dtype == torch.float32 else capi.FDBB_F64
    stream = torch.cuda.current_stream(DEV).cuda_stream
    U0 = [[torch.from_numpy(u).to(DEV).to(dtype) for u in _initial(n, 40 + i)] for i, n in enumerate(sizes)]

    # reference: caller-owned scratch, three slots per grid
    smax = torch.zeros(3 * len(sizes), dtype=dtype, device=DEV)
    ref = [fv.grid_from_conservative(U, n, i, smax, G_, dt_log_steps=steps) for i, (n, U) in enumerate(zip(sizes, U0))]
    for _ in range(steps):
        fv.rusanov_step(ref, smax, G_, CFL)

    # allocation-free entry point, two calls in a row
    grids = []
    for n, U in zip(sizes, U0):
        g = fv.FvGrid([u.clone() for u in U], [torch.empty_like(u) for u in U], n, slot=12345,
                      dt_log=torch.zeros(steps, dtype=torch.float64, device=DEV))
        g.phase = 2  # ignored by the entry point
        grids.append(g)
    free = []
    for _ in range(steps):
        tab, vcells = fv._table(grids, with_new=True)
        capi.call("fdbb_fv_rusanov_step_noalloc", len(grids), tab, vcells, G_, CFL, code, stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info(DEV)[0])
        for g in grids:
            g.advance()
    torch.cuda.synchronize()
    # the second call (after the first has loaded the kernels and looked up
    # the array's address) leaves the device's free memory as it was
    assert free[1] == free[0]

    for i, (a, b) in enumerate(zip(ref, grids)):
        assert a.step == b.step == steps
        assert torch.equal(b.dt_log, a.dt_log), i
        for k in range(5):
            assert torch.equal(a.U[k], b.U[k]), (i, k)
    # and against the FP64 oracle, from the same (stored-precision) start
    for i, (n, b) in enumerate(zip(sizes, grids)):
        start = [u.double().cpu().numpy() for u in U0[i]]
        want, dts = oracle.rusanov_run(n, G_, CFL, steps, start)
        np.testing.assert_allclose(b.dt_log.cpu().numpy(), dts, rtol=TOL[dtype])
        for k in range(5):
            got = b.U[k].double().cpu().numpy()
            assert np.abs(got - want[k]).max() <= TOL[dtype] * max(1.0, np.abs(want[k]).max()), (i, k)


def test_noalloc_rejects_more_grids_than_its_array_holds():
    build.build()
    L = capi.lib()
    tab = (capi.FvGrid * 1)()
    st = L.fdbb_fv_rusanov_step_noalloc(capi.FV_MAX_GRIDS + 1, tab, 0, G_, CFL, capi.FDBB_F32, None)
    assert st == 1  # FDBB_ERR_ARG, before any launch
