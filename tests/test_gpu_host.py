"""Fields in pinned host memory: fdbb_pointer_kind, fdbb_euler_fused_host and
the three modes of blocks.euler_fused_host give the device results bit for
bit; memory the device cannot reach is rejected before any launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_09851_gb300 import blocks, capi, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_09851_gb300 import build
    build.build()
    capi.lib()
    assert torch.cuda.is_available()


def _fields(n, seed=3):
    V = synth.euler3d(n, seed=seed)
    U = oracle.cons_from_prim(3, 1.4, V)
    W = synth.char_weights(n, 5, seed=seed + 1)
    return [torch.from_numpy(u).to(DEV) for u in U], [torch.from_numpy(w).to(DEV) for w in W]


def _pinned(rows, n, dtype=torch.float64):
    """Pinned (rows, n) planes, each row starting on a 16-byte boundary."""
    pad = -(-n // 2) * 2
    h = torch.empty(rows, pad, dtype=dtype, pin_memory=True)[:, :n]
    return h, list(h.unbind(0))


def test_pointer_kinds():
    L = capi.lib()
    d = torch.empty(64, dtype=torch.float64, device=DEV)
    h = torch.empty(64, dtype=torch.float64, pin_memory=True)
    p = torch.empty(64, dtype=torch.float64)
    assert L.fdbb_pointer_kind(d.data_ptr()) == capi.FDBB_PTR_DEVICE
    assert L.fdbb_pointer_kind(d[8:].data_ptr()) == capi.FDBB_PTR_DEVICE
    assert L.fdbb_pointer_kind(h.data_ptr()) == capi.FDBB_PTR_HOST
    assert L.fdbb_pointer_kind(h[16:].data_ptr()) == capi.FDBB_PTR_HOST
    assert L.fdbb_pointer_kind(p.data_ptr()) == capi.FDBB_PTR_OTHER
    assert L.fdbb_pointer_kind(None) == capi.FDBB_PTR_OTHER


@pytest.mark.parametrize("dw", [False, True], ids=["f64", "f64dw"])
@pytest.mark.parametrize("n", [1, 1000, (1 << 20) + 3])
def test_fused_host_planes_match_device(n, dw):
    U, W = _fields(n)
    F, A, Y = blocks.euler_fused(U, W, 1, 1.4, dw=dw)
    ref = F + A + Y
    hI, ri = _pinned(10, n)
    for k, t in enumerate(U + W):
        ri[k].copy_(t)
    hO, ro = _pinned(45, n)
    # inputs on the host (direct kernel), outputs on the host
    blocks.euler_fused_mapped(ri[:5], ri[5:], (ro[:15], ro[15:40], ro[40:]), 1, 1.4, dw=dw)
    torch.cuda.synchronize()
    for k in range(45):
        assert torch.equal(hO[k], ref[k].cpu()), k
    # inputs on the device (staged kernel for large n), outputs on the host
    hO.zero_()
    blocks.euler_fused_mapped(U, W, (ro[:15], ro[15:40], ro[40:]), 1, 1.4, dw=dw)
    torch.cuda.synchronize()
    for k in range(45):
        assert torch.equal(hO[k], ref[k].cpu()), k


@pytest.mark.parametrize("mode", ["mapped_out", "mapped", "copy"])
def test_host_pipeline_modes(mode):
    n = 3 * (1 << 18) + 77  # several chunks and a ragged last one
    U, W = _fields(n, seed=8)
    F, A, Y = blocks.euler_fused(U, W, 0, 1.4, dw=True)
    ref = F + A + Y
    hI, ri = _pinned(10, n)
    for k, t in enumerate(U + W):
        ri[k].copy_(t)
    hO, ro = _pinned(45, n)
    work = None
    for _ in range(2):  # the second call reuses the staging buffers
        hO.zero_()
        work = blocks.euler_fused_host(ri[:5], ri[5:], (ro[:15], ro[15:40], ro[40:]), 0, 1.4, chunk=1 << 18,
                                       dw=True, mode=mode, work=work)
        torch.cuda.synchronize()
        for k in range(45):
            assert torch.equal(hO[k], ref[k].cpu()), (mode, k)


def test_unreachable_memory_is_rejected_before_launch():
    n = 4096
    U, W = _fields(n)
    pageable = [torch.zeros(n, dtype=torch.float64) for _ in range(45)]
    pl = lambda ts: capi.planes([t.data_ptr() for t in ts])
    L = capi.lib()
    # pageable host outputs
    st = L.fdbb_euler_fused_host(3, 0, 1.4, n, capi.FDBB_F64, pl(U), pl(W), pl(pageable[:15]), pl(pageable[15:40]),
                                 pl(pageable[40:]), None)
    assert st == 1  # FDBB_ERR_ARG
    # a pageable input plane
    Ubad = [pageable[0]] + U[1:]
    dO = [torch.empty(n, dtype=torch.float64, device=DEV) for _ in range(45)]
    st = L.fdbb_euler_fused_host(3, 0, 1.4, n, capi.FDBB_F64, pl(Ubad), pl(W), pl(dO[:15]), pl(dO[15:40]),
                                 pl(dO[40:]), None)
    assert st == 1
    torch.cuda.synchronize()
    assert all(float(t.abs().sum()) == 0.0 for t in pageable)
