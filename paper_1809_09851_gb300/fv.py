"""Batched Rusanov finite-volume steps on periodic n^3 grids (binding).

Thin marshalling over ``fdbb_fv_max_speed`` / ``fdbb_fv_rusanov_step``
(include/fdbb.h): a list of :class:`FvGrid` states is laid out in the virtual
cell index space (each grid padded to a multiple of the 256-cell tile),
packed into descriptor tables of at most 256 grids and advanced by one
launch per table.  The per-grid wave-speed scratch ``smax`` (three slots per
grid, storage dtype) is owned by the caller.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch

from . import blocks, capi

TILE = capi.FV_TILE
MAX_GRIDS = capi.FV_MAX_GRIDS
_CODES = {torch.float32: capi.FDBB_F32, torch.float64: capi.FDBB_F64}


def padded_cells(n: int) -> int:
    return (n ** 3 + TILE - 1) // TILE * TILE


class FvGrid:
    """State of one periodic n^3 grid: U (current), Unew (next), its
    wave-speed slot, the step index and the step phase (step mod 3)."""

    def __init__(self, U: List[torch.Tensor], Unew: List[torch.Tensor], n: int, slot: int,
                 dt_log: Optional[torch.Tensor] = None):
        self.U, self.Unew, self.n, self.slot = list(U), list(Unew), n, slot
        self.phase = 0
        self.step = 0
        self.dt_log = dt_log

    @property
    def dtype(self):
        return self.U[0].dtype

    def advance(self):
        self.U, self.Unew = self.Unew, self.U
        self.phase = (self.phase + 1) % 3
        self.step += 1


def _table(grids: Sequence[FvGrid], with_new: bool):
    arr = (capi.FvGrid * max(1, len(grids)))()
    off = 0
    for i, g in enumerate(grids):
        e = arr[i]
        for q in range(5):
            e.U[q] = g.U[q].data_ptr()
            e.Unew[q] = g.Unew[q].data_ptr() if with_new else None
        e.dt_log = g.dt_log.data_ptr() if g.dt_log is not None else None
        e.cell_begin = off
        e.n, e.slot, e.phase, e.step = g.n, g.slot, g.phase, g.step
        off += padded_cells(g.n)
    return arr, off


def _chunks(grids):
    for i in range(0, len(grids), MAX_GRIDS):
        yield grids[i:i + MAX_GRIDS]


def _stream(stream, device) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


def max_speed(grids: Sequence[FvGrid], smax: torch.Tensor, gamma: float = 1.4, stream=None):
    """Reduce max sum_d(|v_d| + c) of each grid's U into smax[3*slot + phase]
    (the slot must be zero)."""
    if not grids:
        return
    code = _CODES[grids[0].dtype]
    for ch in _chunks(list(grids)):
        tab, vcells = _table(ch, with_new=False)
        capi.call("fdbb_fv_max_speed", len(ch), tab, vcells, gamma, code, smax.data_ptr(),
                  _stream(stream, smax.device))


def rusanov_step(grids: Sequence[FvGrid], smax: torch.Tensor, gamma: float = 1.4, cfl: float = 0.4,
                 stream=None):
    """Advance every grid by one step (one launch per 256 grids)."""
    if not grids:
        return
    code = _CODES[grids[0].dtype]
    for ch in _chunks(list(grids)):
        tab, vcells = _table(ch, with_new=True)
        capi.call("fdbb_fv_rusanov_step", len(ch), tab, vcells, gamma, cfl, code, smax.data_ptr(),
                  _stream(stream, smax.device))
    for g in grids:
        g.advance()


def new_grid(V: Sequence[torch.Tensor], n: int, slot: int, smax: torch.Tensor, gamma: float = 1.4,
             dt_log_steps: int = 0, stream=None) -> FvGrid:
    """Allocate U/Unew, convert the primitive planes V to conservative U with
    fdbb_cons_from_prim, clear the grid's three wave-speed slots and reduce the
    initial wave speed into slot 0."""
    dtype, device = V[0].dtype, V[0].device
    cells = n ** 3
    U = [torch.empty(cells, dtype=dtype, device=device) for _ in range(5)]
    Unew = [torch.empty(cells, dtype=dtype, device=device) for _ in range(5)]
    with torch.cuda.stream(stream) if stream is not None else _null():
        blocks.cons_from_prim(list(V), gamma, out=U, stream=stream)
        smax[3 * slot:3 * slot + 3].zero_()
    dt_log = torch.zeros(dt_log_steps, dtype=torch.float64, device=device) if dt_log_steps else None
    g = FvGrid(U, Unew, n, slot, dt_log)
    max_speed([g], smax, gamma, stream)
    return g


def new_grid_smooth(n: int, seed: int, slot: int, smax: torch.Tensor, dtype, device, gamma: float = 1.4,
                    amplitude: float = 0.1, dt_log_steps: int = 0, stream=None) -> FvGrid:
    """A grid holding the smooth seeded initial state of a serving request
    (the data of synth.smooth_perturbation, built on the device by
    fdbb_fv_init_smooth in two launches), with its wave-speed slots cleared
    and the initial wave speed reduced into slot 0."""
    import numpy as np

    from . import synth
    cells = n ** 3
    U = [torch.empty(cells, dtype=dtype, device=device) for _ in range(5)]
    Unew = [torch.empty(cells, dtype=dtype, device=device) for _ in range(5)]
    wave = np.empty(30, dtype=np.float64)
    for r, (k, ph, a) in enumerate(synth.smooth_params(seed)):
        for m in range(3):
            wave[15 * r + 5 * m: 15 * r + 5 * m + 5] = (k[m, 0], k[m, 1], k[m, 2], ph[m], a[m])
    scratch = torch.empty(2, dtype=dtype, device=device)
    dt_log = torch.zeros(dt_log_steps, dtype=torch.float64, device=device) if dt_log_steps else None
    g = FvGrid(U, Unew, n, slot, dt_log)
    tab, _ = _table([g], with_new=False)
    s = _stream(stream, device)
    capi.call("fdbb_fv_init_smooth", tab, gamma, amplitude, wave.ctypes.data, _CODES[dtype], scratch.data_ptr(), s)
    with torch.cuda.stream(stream) if stream is not None else _null():
        smax[3 * slot:3 * slot + 3].zero_()
    max_speed([g], smax, gamma, stream)
    return g


class FvSnapshot:
    """A grid's state in host memory: its conservative planes, the steps it
    has taken and, if it logs them, its time steps so far."""

    def __init__(self, n: int, step: int, U: List[torch.Tensor], dt_log: Optional[torch.Tensor]):
        self.n, self.step, self.U, self.dt_log = n, step, U, dt_log


def snapshot(g: FvGrid, stream=None) -> FvSnapshot:
    """Copy a grid's state to host memory once the work queued on `stream`
    (default: the current stream) has run; blocks until the copy is done."""
    s = stream if stream is not None else torch.cuda.current_stream(g.U[0].device)
    s.synchronize()
    U = [u.to("cpu") for u in g.U]
    dt = g.dt_log.to("cpu") if g.dt_log is not None else None
    return FvSnapshot(g.n, g.step, U, dt)


def restore(snap: FvSnapshot, slot: int, smax: torch.Tensor, gamma: float = 1.4, dt_log_steps: int = 0,
            stream=None) -> FvGrid:
    """A grid that resumes from a snapshot: its planes back on the device, its
    step count, its logged time steps, its wave-speed slot reduced afresh from
    the state (the exact maximum the step kernel would have left there, so the
    resumed steps are bit for bit those of an uninterrupted run)."""
    device = smax.device
    U = [u.to(device) for u in snap.U]
    g = grid_from_conservative(U, snap.n, slot, smax, gamma, dt_log_steps=dt_log_steps, stream=stream)
    g.step = snap.step
    if g.dt_log is not None and snap.dt_log is not None:
        k = min(snap.dt_log.numel(), g.dt_log.numel())
        g.dt_log[:k].copy_(snap.dt_log[:k])
    return g


class _null:
    def __enter__(self):
        return None

    def __exit__(self, *a):
        return False


def grid_from_conservative(U: Sequence[torch.Tensor], n: int, slot: int, smax: torch.Tensor,
                           gamma: float = 1.4, dt_log_steps: int = 0, stream=None) -> FvGrid:
    """Like new_grid, from conservative planes (copied)."""
    dtype, device = U[0].dtype, U[0].device
    Uc = [u.clone() for u in U]
    Unew = [torch.empty_like(u) for u in U]
    smax[3 * slot:3 * slot + 3].zero_()
    dt_log = torch.zeros(dt_log_steps, dtype=torch.float64, device=device) if dt_log_steps else None
    g = FvGrid(Uc, Unew, n, slot, dt_log)
    max_speed([g], smax, gamma, stream)
    return g
