"""Failure path of the staged kernels' bounded waits, without a GPU fault.

The staged kernel waits on an mbarrier for the bulk copies of each input tile
with a bounded number of polls.  fdbb_set_wait_limit(0) makes every such wait
give up at once: each block counts the event, waits (with the default limit)
for the copies it has issued so that none lands after it exits, and returns
without writing.  The host then reads FDBB_ERR_TIMEOUT from
fdbb_device_status, the context stays usable, and the next call with the
default limit is correct.  Nothing here faults, traps or hangs the device.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_09851_gb300 import blocks, build, capi, synth

pytestmark = pytest.mark.gpu
G = 1.4
DEV = "cuda:0"
SENTINEL = 12345.0


def _field(n):
    U = oracle.cons_from_prim(3, G, synth.euler3d(n, seed=606))
    W = synth.char_weights(n, 5, seed=607)
    return U, W


def _staged_n(tile, tail):
    return 4 * torch.cuda.get_device_properties(DEV).multi_processor_count * tile + tail


@pytest.fixture(autouse=True)
def _restore_limit():
    build.build()
    L = capi.lib()
    capi.device_status()  # clear earlier counts
    prev = L.fdbb_set_wait_limit(-1)
    yield L
    L.fdbb_set_wait_limit(prev)
    capi.CHECK_DEVICE = False


def test_wait_that_runs_out_is_reported_and_writes_nothing(_restore_limit):
    L = _restore_limit
    n = _staged_n(512, 7)  # the double-word fused pass takes 512-point tiles (two points per thread)
    U, W = _field(n)
    Ud = [torch.from_numpy(u).to(DEV) for u in U]
    Wd = [torch.from_numpy(w).to(DEV) for w in W]
    out = tuple([torch.full((n,), SENTINEL, dtype=torch.float64, device=DEV) for _ in range(k)] for k in (15, 25, 5))
    L.fdbb_set_wait_limit(0)
    blocks.euler_fused(Ud, Wd, 0, G, out=out, dw=True)
    assert capi.last_launch().kernel == capi.FDBB_KERNEL_STAGED
    st = capi.device_status()
    L.fdbb_set_wait_limit(-1)
    assert st == capi.STATUS_CODES["FDBB_ERR_TIMEOUT"]
    for t in (*out[0], *out[1], *out[2]):
        assert bool((t == SENTINEL).all())  # every block gave up before writing
    # the count was cleared by the read, and the context is still usable: the
    # same call with the default limit is correct
    assert capi.device_status() == 0
    F, A, Y = blocks.euler_fused(Ud, Wd, 0, G, out=out, dw=True)
    assert capi.last_launch().kernel == capi.FDBB_KERNEL_STAGED
    assert capi.device_status() == 0
    ref, S = oracle.euler_fused(3, 0, G, U, W, scale=True)
    for k, (g, o, s) in enumerate(zip([t.cpu().numpy() for t in (*F, *A, *Y)], ref, S)):
        assert np.all(np.abs(g - o) <= 1e-12 * s), k


def test_python_check_raises_on_a_wait_that_ran_out(_restore_limit):
    L = _restore_limit
    n = _staged_n(512, 3)  # IEEE-double flux: 512-point tiles
    U, _ = _field(n)
    Ud = [torch.from_numpy(u).to(DEV) for u in U]
    capi.CHECK_DEVICE = True
    L.fdbb_set_wait_limit(0)
    with pytest.raises(capi.FdbbError) as e:
        blocks.flux(Ud, 0, G)
    L.fdbb_set_wait_limit(-1)
    assert e.value.status == capi.STATUS_CODES["FDBB_ERR_TIMEOUT"]
    F = blocks.flux(Ud, 0, G)  # checked again, with the default limit: no error
    capi.CHECK_DEVICE = False
    ref = oracle.flux(3, 0, G, U)
    for g, o in zip(F, ref):
        np.testing.assert_allclose(g.cpu().numpy(), o, rtol=1e-12, atol=1e-300)


def test_direct_kernel_is_untouched_by_the_limit(_restore_limit):
    """The direct kernel has no waits: a small call is correct under limit 0."""
    L = _restore_limit
    n = 4099
    U, _ = _field(n)
    Ud = [torch.from_numpy(u).to(DEV) for u in U]
    L.fdbb_set_wait_limit(0)
    p, c = blocks.eos(Ud, G)
    assert capi.last_launch().kernel == capi.FDBB_KERNEL_DIRECT
    L.fdbb_set_wait_limit(-1)
    assert capi.device_status() == 0
    (pr, cr), (Sp, Sc) = oracle.eos(3, G, U, scale=True)
    assert np.all(np.abs(p.cpu().numpy() - pr) <= 1e-12 * Sp)
    assert np.all(np.abs(c.cpu().numpy() - cr) <= 1e-12 * Sc)
