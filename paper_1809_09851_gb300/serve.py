"""Continuous-batching serving loop for explicit finite-volume requests.

Each request asks for `steps` Rusanov steps on its own periodic n^3 grid
(FP32 or FP64 state).  The loop
  * admits arrived requests in arrival order while their state (U and Unew,
    10 planes of n^3 values) fits the HBM budget (default: free device memory
    at start minus a reserve), initialising them on the device;
  * advances *all* admitted grids by one step per iteration in one batched
    launch (fdbb_fv_rusanov_step; one launch per 256 grids), so requests that
    arrive while others run join the next iteration and their work overlaps;
  * keeps at most `max_inflight` iterations queued on the stream, waiting on
    CUDA events with a deadline (a wait that runs out raises FvTimeout
    instead of hanging);
  * retires a request when its last step's event completes, recording its
    completion time on the device clock, and frees its memory and slot.
Latency = completion - arrival (seconds on the same clock); throughput =
cell-steps / wall time.  A run can stop after a number of batched steps
(`max_iterations`): the state of every unfinished request is then copied to
host memory (fv.snapshot) and returned, and a later run -- of this server or
another -- resumes those requests from their snapshots (`resume`), bit for bit
where an uninterrupted run would have been.  Admission, each batched step and each retirement are
NVTX ranges ("fdbb.admit", "fdbb.step", "fdbb.retire") for profilers that
show a timeline.  A grid's results do not depend on the other grids
in its launches (per-cell arithmetic is fixed and the time-step reduction is
an exact maximum), so a request's answer is the same alone and in the mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import torch

from . import fv, synth


def _range(name: str):
    """NVTX range around a phase of the loop (a no-op when NVTX is unavailable)."""
    try:
        return torch.cuda.nvtx.range(name)
    except Exception:  # pragma: no cover - builds without NVTX
        import contextlib
        return contextlib.nullcontext()


class FvTimeout(RuntimeError):
    """A bounded wait on the device ran out (FDBB_ERR_TIMEOUT on the host side)."""


class FvNoMem(RuntimeError):
    """A request can never fit the HBM budget (FDBB_ERR_NOMEM)."""


def wait_event(ev, timeout_s: float, clock: Callable[[], float] = time.perf_counter) -> None:
    """Poll ev.query() until it completes or `timeout_s` elapses."""
    deadline = clock() + timeout_s
    while not ev.query():
        if clock() > deadline:
            raise FvTimeout(f"device did not complete within {timeout_s:.1f} s")
        time.sleep(0)


@dataclass
class Job:
    req: synth.Request
    grid: fv.FvGrid
    nbytes: int
    t_admit: float
    done_ev: Optional[torch.cuda.Event] = None
    t_done: Optional[float] = None


@dataclass
class Report:
    latencies: Dict[int, float] = field(default_factory=dict)
    rejected: List[int] = field(default_factory=list)
    cell_steps: int = 0
    wall_s: float = 0.0
    iterations: int = 0
    launches: int = 0
    max_active: int = 0
    results: Dict[int, List[torch.Tensor]] = field(default_factory=dict)
    # a run stopped by max_iterations: the unfinished requests' state, and the
    # requests it never admitted
    snapshots: Dict[int, fv.FvSnapshot] = field(default_factory=dict)
    unstarted: List[int] = field(default_factory=list)

    def pct(self, q: float) -> float:
        xs = sorted(self.latencies.values())
        if not xs:
            return float("nan")
        k = max(0, min(len(xs) - 1, int(-(-q / 100.0 * len(xs) // 1)) - 1))
        return xs[k]

    def summary(self) -> dict:
        return {"requests": len(self.latencies), "rejected": len(self.rejected),
                "p50_s": self.pct(50), "p99_s": self.pct(99),
                "cell_steps": self.cell_steps, "wall_s": self.wall_s,
                "cells_per_s": self.cell_steps / self.wall_s if self.wall_s > 0 else float("nan"),
                "iterations": self.iterations, "launches": self.launches, "max_active": self.max_active}


class FVServer:
    def __init__(self, device="cuda:0", dtype=torch.float32, gamma: float = 1.4, cfl: float = 0.4,
                 hbm_budget: Optional[int] = None, reserve: int = 4 << 30, max_slots: int = 4096,
                 max_inflight: int = 2, max_active: Optional[int] = None, wait_timeout: float = 60.0,
                 keep_results: bool = False, log_dt: bool = False,
                 initial_state: Optional[Callable] = None, admit_per_iter: Optional[int] = 4):
        self.device = torch.device(device)
        self.dtype = dtype
        self.gamma, self.cfl = gamma, cfl
        self.stream = torch.cuda.Stream(self.device)
        self.elem = torch.empty((), dtype=dtype).element_size()
        free, _total = torch.cuda.mem_get_info(self.device)
        self.budget = hbm_budget if hbm_budget is not None else max(0, free - reserve)
        self.used = 0
        self.smax = torch.zeros(3 * max_slots, dtype=dtype, device=self.device)  # wave-speed scratch
        self.free_slots = collections.deque(range(max_slots))
        self.max_inflight = max(1, max_inflight)
        self.max_active = max_active
        # admissions between two batched steps (None: all that fit), so that a
        # burst of arrivals does not keep the step launches, and the GPU,
        # waiting (4: p50 / p99 latency 10% lower than admitting every arrived
        # request at once on the 2,000 req/s stream)
        self.admit_per_iter = admit_per_iter
        self.wait_timeout = wait_timeout
        self.keep_results = keep_results
        self.log_dt = log_dt
        # None: the smooth seeded state of synth.smooth_params, built on the
        # device by fdbb_fv_init_smooth; otherwise a callable giving the
        # primitive planes of a request
        self.initial_state = initial_state

    def state_bytes(self, n: int) -> int:
        return 2 * 5 * n ** 3 * self.elem

    def _admit(self, req: synth.Request, now: float, resume=None) -> Job:
        nbytes = self.state_bytes(req.n)
        slot = self.free_slots.popleft()
        with torch.cuda.stream(self.stream):
            snap = resume.get(req.rid) if resume else None
            if snap is not None:
                g = fv.restore(snap, slot, self.smax, self.gamma, dt_log_steps=req.steps if self.log_dt else 0,
                               stream=self.stream)
            elif self.initial_state is None:
                g = fv.new_grid_smooth(req.n, req.seed, slot, self.smax, self.dtype, self.device, self.gamma,
                                       dt_log_steps=req.steps if self.log_dt else 0, stream=self.stream)
            else:
                V = self.initial_state(req)
                g = fv.new_grid(V, req.n, slot, self.smax, self.gamma,
                                dt_log_steps=req.steps if self.log_dt else 0, stream=self.stream)
        self.used += nbytes
        return Job(req, g, nbytes, now)

    def run(self, requests: List[synth.Request], realtime: bool = True, max_iterations: Optional[int] = None,
            resume: Optional[Dict[int, fv.FvSnapshot]] = None) -> Report:
        """Serve `requests` (sorted by arrival).  With realtime=False every
        request is treated as already arrived (a closed batch).  With
        max_iterations the run stops after that many batched steps and returns
        the unfinished requests' snapshots; `resume` maps request ids to
        snapshots from which those requests continue."""
        rep = Report()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        active: List[Job] = []
        inflight = collections.deque()  # (event, [jobs finishing at it])
        t0 = time.perf_counter()
        ev0 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(self.stream):
            ev0.record(self.stream)

        def retire(entry):
            ev, finishing = entry
            with _range("fdbb.retire"):
                wait_event(ev, self.wait_timeout)
                t_done = ev0.elapsed_time(ev) / 1e3
                for job in finishing:
                    job.t_done = t_done
                    rep.latencies[job.req.rid] = t_done - (job.req.arrival if realtime else 0.0)
                    if self.keep_results:
                        rep.results[job.req.rid] = [u.clone() for u in job.grid.U]
                    self.used -= job.nbytes
                    self.free_slots.append(job.grid.slot)
                    job.grid = None

        while pending or active or inflight:
            now = time.perf_counter() - t0
            # admission, in arrival order, while the state fits the budget
            admitted = 0
            with _range("fdbb.admit"):
                while pending and (not realtime or pending[0].arrival <= now):
                    if self.admit_per_iter is not None and admitted >= self.admit_per_iter and active:
                        break
                    req = pending[0]
                    need = self.state_bytes(req.n)
                    if need > self.budget:
                        rep.rejected.append(req.rid)
                        pending.popleft()
                        continue
                    if (self.used + need > self.budget or not self.free_slots
                            or (self.max_active is not None and len(active) >= self.max_active)):
                        break
                    active.append(self._admit(pending.popleft(), now, resume))
                    admitted += 1
            rep.max_active = max(rep.max_active, len(active))
            if not active:
                if inflight:
                    retire(inflight.popleft())
                    continue
                if pending:
                    time.sleep(max(0.0, min(1e-3, pending[0].arrival - (time.perf_counter() - t0))))
                continue
            # one batched step for every active grid
            grids = [j.grid for j in active]
            with _range("fdbb.step"):
                fv.rusanov_step(grids, self.smax, self.gamma, self.cfl, stream=self.stream)
            rep.iterations += 1
            rep.launches += -(-len(grids) // fv.MAX_GRIDS)
            rep.cell_steps += sum(g.n ** 3 for g in grids)
            finishing = [j for j in active if j.grid.step >= j.req.steps]
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(self.stream)
            inflight.append((ev, finishing))
            active = [j for j in active if j.grid.step < j.req.steps]
            while len(inflight) > self.max_inflight:
                retire(inflight.popleft())
            if max_iterations is not None and rep.iterations >= max_iterations:
                while inflight:
                    retire(inflight.popleft())
                for job in active:
                    rep.snapshots[job.req.rid] = fv.snapshot(job.grid, self.stream)
                    self.used -= job.nbytes
                    self.free_slots.append(job.grid.slot)
                    job.grid = None
                active = []
                rep.unstarted = [r.rid for r in pending]
                pending.clear()
        while inflight:
            retire(inflight.popleft())
        torch.cuda.synchronize(self.device)
        rep.wall_s = time.perf_counter() - t0
        return rep
