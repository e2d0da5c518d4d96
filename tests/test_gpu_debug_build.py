"""The debug build (libfdbb_debug.so, compiled with -DFDBB_DEBUG): its kernels
check every global-memory index against the field's size, and every plane
index of the staged kernels' shared-memory ring, before each access,
recording violations instead of trapping.  The point-wise blocks (direct and
staged kernels, ragged tails, packed double-word pairs, every storage form)
and the finite-volume steps (FP32 and FP64, scratch-using and
allocation-free) run under it with no violation and with the results of the
release build.  The debug library loads in a child process (FDBB_DEBUG=1)."""
import os
import subprocess
import sys

import pytest

from paper_1809_09851_gb300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle
from paper_1809_09851_gb300 import blocks, capi, fv, synth
assert capi.LIBRARY.endswith("libfdbb_debug.so"), capi.LIBRARY
dev = "cuda:0"
G = 1.4
assert capi.debug_index_faults()[0] == 0
sms = torch.cuda.get_device_properties(dev).multi_processor_count
for n in (1, 7, 4099, 4 * sms * 1024 + 4103):
    U = oracle.cons_from_prim(3, G, synth.euler3d(n, seed=71))
    W = synth.char_weights(n, 5, seed=72)
    for dt, dw in ((torch.float64, True), (torch.float64, False), (torch.float32, False), (torch.bfloat16, False)):
        Ud = [torch.from_numpy(u).to(dev).to(dt) for u in U]
        Wd = [torch.from_numpy(w).to(dev).to(dt) for w in W]
        F, A, Y = blocks.euler_fused(Ud, Wd, 1, G, dw=dw)
        blocks.eos(Ud, G, dw=dw)
        blocks.prim_from_cons(Ud, G, dw=dw)
        blocks.flux_vjp(Ud, Wd, 0, G, dw=dw)
        blocks.char_transform(Ud, Wd, 2, G, inverse=True, dw=dw)
        blocks.roe_flux(Ud, [torch.roll(u, 1) for u in Ud], 0, G, dw=dw)
        if dt == torch.float64:
            ref, S = oracle.euler_fused(3, 1, G, U, W, scale=True)
            for g, o, s in zip([t.cpu().numpy() for t in (*F, *A, *Y)], ref, S):
                assert np.all(np.abs(g - o) <= 1e-12 * s)
torch.cuda.synchronize()
for dt in (torch.float32, torch.float64):
    smax = torch.zeros(3 * 3, dtype=dt, device=dev)
    grids = [fv.new_grid_smooth(m, 5 + m, i, smax, dt, dev) for i, m in enumerate((5, 33, 40))]
    for _ in range(3):
        fv.rusanov_step(grids, smax)
    tab, vcells = fv._table(grids, with_new=True)
    code = capi.FDBB_F32 if dt == torch.float32 else capi.FDBB_F64
    capi.call("fdbb_fv_rusanov_step_noalloc", len(grids), tab, vcells, G, 0.4, code,
              torch.cuda.current_stream(dev).cuda_stream)
torch.cuda.synchronize()
count, first = capi.debug_index_faults()
assert capi.device_status() == 0
print("index violations", count, "first", first)
assert (count, first) == (0, -1), (count, first)
"""


def test_debug_build_kernels_record_no_index_violation():
    build.build(debug=True)
    env = dict(os.environ, FDBB_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "index violations 0 first -1" in r.stdout
