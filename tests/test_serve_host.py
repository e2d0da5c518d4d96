"""Host-side checks of the finite-volume ABI and serving loop (no GPU):
argument validation before any launch, and bounded waits that time out."""
import pytest

from paper_1809_09851_gb300 import build as lib_build
from paper_1809_09851_gb300 import capi

A = 1 << 20


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return capi.lib()


def _grid(n=4, begin=0, slot=0, base=A, new_base=A + (1 << 16)):
    g = capi.FvGrid()
    for q in range(5):
        g.U[q] = base + 4096 * q
        g.Unew[q] = new_base + 4096 * q
    g.cell_begin, g.n, g.slot, g.phase, g.step = begin, n, slot, 0, 0
    return g


def _tab(*gs):
    arr = (capi.FvGrid * len(gs))(*gs)
    return arr


def test_fv_argument_errors(L):
    F32, F16 = capi.FDBB_F32, capi.FDBB_F16
    ok = _tab(_grid(4, 0), _grid(4, 256, 1, base=A + (1 << 18), new_base=A + (1 << 19)))
    step = L.fdbb_fv_rusanov_step
    # vcells not a tile multiple / too small for the ranges
    assert step(2, ok, 300, 1.4, 0.4, F32, A, None) == 1
    assert step(2, ok, 256, 1.4, 0.4, F32, A, None) == 1
    # unsorted / overlapping ranges
    assert step(2, _tab(_grid(4, 256), _grid(4, 0, 1)), 512, 1.4, 0.4, F32, A, None) == 1
    assert step(2, _tab(_grid(9, 0), _grid(4, 256, 1)), 2048, 1.4, 0.4, F32, A, None) == 1
    # Unew aliases U
    assert step(1, _tab(_grid(4, 0, new_base=A)), 256, 1.4, 0.4, F32, A, None) == 1
    # storage type, misaligned scratch, NULL scratch, bad cfl, too many grids
    assert step(2, ok, 512, 1.4, 0.4, F16, A, None) == 4
    assert step(2, ok, 512, 1.4, 0.4, F32, A + 2, None) == 3
    assert step(2, ok, 512, 1.4, 0.4, F32, None, None) == 2
    assert step(2, ok, 512, 1.4, -1.0, F32, A, None) == 1
    assert step(257, ok, 512, 1.4, 0.4, F32, A, None) == 1
    # an empty batch is a no-op
    assert step(0, None, 0, 1.4, 0.4, F32, None, None) == 0
    assert L.fdbb_fv_max_speed(0, None, 0, 1.4, F32, None, None) == 0


def test_wait_event_times_out():
    from paper_1809_09851_gb300 import serve

    class Never:
        def query(self):
            return False

    t = [0.0]

    def clock():
        t[0] += 0.25
        return t[0]

    with pytest.raises(serve.FvTimeout):
        serve.wait_event(Never(), 1.0, clock=clock)

    class Done:
        def query(self):
            return True

    serve.wait_event(Done(), 1.0)


def test_noalloc_checks_arguments_before_any_cuda_call(L):
    """The allocation-free step validates its grid table before it looks up
    its device array: on a host without a GPU (where any CUDA call fails) bad
    tables still give their argument errors, and an empty batch is a no-op."""
    F32, F16 = capi.FDBB_F32, capi.FDBB_F16
    step = L.fdbb_fv_rusanov_step_noalloc
    ok = _tab(_grid(4, 0), _grid(4, 256, 1, base=A + (1 << 18), new_base=A + (1 << 19)))
    assert step(2, ok, 300, 1.4, 0.4, F32, None) == 1                     # vcells not a tile multiple
    assert step(2, _tab(_grid(4, 256), _grid(4, 0, 1)), 512, 1.4, 0.4, F32, None) == 1  # unsorted
    assert step(1, _tab(_grid(4, 0, new_base=A)), 256, 1.4, 0.4, F32, None) == 1       # Unew aliases U
    assert step(2, ok, 512, 1.4, 0.4, F16, None) == 4                     # storage type
    assert step(1, _tab(_grid(4, 0, base=A + 2)), 256, 1.4, 0.4, F32, None) == 3       # misaligned plane
    assert step(2, ok, 512, 1.4, 0.0, F32, None) == 1                     # cfl
    assert step(capi.FV_MAX_GRIDS + 1, ok, 512, 1.4, 0.4, F32, None) == 1  # beyond the array
    assert step(0, None, 0, 1.4, 0.4, F32, None) == 0
