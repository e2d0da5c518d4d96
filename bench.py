#!/usr/bin/env python3
"""Benchmark: fused 3D Euler building blocks on GB300.

One step = one fdbb_euler_fused launch over N = 2^26 points of a 3D field:
reads U (5 planes) and W (5 planes), writes F_x, F_y, F_z (15 planes), the
x-Jacobian A_x (25 planes) and L_x(U) W (5 planes) -- 440 B/point in FP64.
The headline value is FP64-storage Gpoints/s in double-word arithmetic (every
output within 1e-12 of the oracle's running-error scale, like IEEE double);
IEEE-double arithmetic, FP32 and BF16 storage are measured on the same field
and reported beside it, then the serving workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fdbb|reference]

With N > 1 (launched by torch.distributed.run) every rank evaluates its own
N-point field (weak scaling, no data-path collective); the time is the max
over ranks and the value is the points of all ranks / that time.

--impl reference times the FP64 CPU oracle on the host cores (rank 0 only)
on a bounded sample of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoints/s & % HBM peak, fused 3D flux+Jacobian, FP64 vs mixed at stated err; p99"
UNIT = "Gpoints/s"
N_POINTS = 1 << 26
GAMMA = 1.4
D = 3
NV = 5
PLANES_IN, PLANES_OUT = 2 * NV, D * NV + NV * NV + NV  # 10 read, 45 written
BYTES = {"f64": 8, "f32": 4, "bf16": 2}
L2_BYTES = 129 * 2 ** 20

# DRAM traffic per point of the fused FP64 kernel from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum per launch / points), valid only
# for the kernel sources whose hash is recorded beside it.
# Measured with ncu on N = 2^22: (335.7 MB read + 1448.7 MB written) / 2^22
# points; scaled to the launch size.
NCU_TRAFFIC = {"source_hash": "f805a5a10623223a", "bytes_per_point": 425.4}


FUSED_KERNEL_SOURCES = ("fdbb_device.cuh", "fdbb_dw.cuh", "fdbb_eos.cuh", "fdbb_kernels.cuh", "fdbb_internal.h",
                        "kern_f64dw3.cu")


def kernel_source_hash(root: str = None) -> str:
    """Hash of the sources that define the headline (fused, double-word) kernel
    (under `root`, default this checkout)."""
    h = hashlib.sha256()
    for p in sorted(os.path.join(root or ROOT, "paper_1809_09851_gb300", "csrc", f) for f in FUSED_KERNEL_SOURCES):
        with open(p, "rb") as fh:
            h.update(os.path.basename(p).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(n: int, root: str = None):
    """DRAM bytes of one headline launch over n points from the recorded ncu
    capture, or None when the kernel sources are no longer the ones it was
    taken on."""
    if not NCU_TRAFFIC["bytes_per_point"] or NCU_TRAFFIC["source_hash"] != kernel_source_hash(root):
        return None
    return round(NCU_TRAFFIC["bytes_per_point"] * n)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            js = json.load(fh)
        return float(js["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_seed(base: int, rank: int) -> int:
    """Each rank evaluates its own independent field."""
    return base + 1000 * rank


SHARD_ALIGN = 256  # points: a rank's range starts on a tile, so its planes stay 16-byte aligned


def shard_bounds(n: int, world: int, rank: int):
    """Contiguous index range [lo, hi) of one n-point field that rank `rank`
    of `world` evaluates when the field is split (the points are independent,
    so the ranks exchange nothing): near-equal shares whose starts are
    multiples of SHARD_ALIGN points; the last rank ends at n."""
    cut = lambda r: n if r >= world else (n * r // world) // SHARD_ALIGN * SHARD_ALIGN
    return cut(rank), cut(rank + 1)


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def make_fields(n, seed, dev, lo=0):
    """Points [lo, lo + n) of the seeded 3D field (U built on the GPU) and W."""
    import torch
    from paper_1809_09851_gb300 import blocks, synth
    V = [torch.from_numpy(v[lo:]).to(dev) for v in synth.euler3d(lo + n, seed=seed)]
    U = blocks.cons_from_prim(V, GAMMA)  # conservative state built on the GPU
    del V
    W = [torch.from_numpy(w[lo:]).to(dev) for w in synth.char_weights(lo + n, NV, seed=seed + 1)]
    return U, W


def time_fused(U, W, out, steps, warmup, stream, dw=False):
    """Per-launch CUDA-event durations (ms) and the wall of the whole timed loop."""
    import torch
    from paper_1809_09851_gb300 import blocks
    F, A, Y = out
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            blocks.euler_fused(U, W, 0, GAMMA, out=(F, A, Y), dw=dw)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for i in range(steps):
            blocks.euler_fused(U, W, 0, GAMMA, out=(F, A, Y), dw=dw)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total = ev[0].elapsed_time(ev[steps])
    return per, total


def time_launch(fn, steps, warmup, stream):
    """Like time_fused, for any launch fn() enqueued on the current stream."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for i in range(steps):
            fn()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)], ev[0].elapsed_time(ev[steps])


def run_general_eos(args, n, W64, out64, stream, dev, world, hbm_peak):
    """The fused 3D pass under the Noble-Abel stiffened-gas EOS (fdbb_euler_fused_eos)
    on the general-EOS workload, FP64 and FP32 storage, same N and planes as the headline."""
    import torch
    from paper_1809_09851_gb300 import blocks, synth
    eos = synth.EOS_NASG
    V = [torch.from_numpy(v).to(dev) for v in synth.euler_eos(n, 3, seed=shard_seed(4242, dist_env()[1]))]
    U = blocks.cons_from_prim_eos(V, eos)
    del V
    res = {"eos": "NASG gamma=1.6 p_inf=1 b=0.1 q=-0.3 c_v=2 (nondimensional)",
           "workload": "rho~U[0.2,4], v~N(0,1), p~U[0.1,10]"}
    for tag, dt, dw in (("f64dw", torch.float64, True), ("f64", torch.float64, False), ("f32", torch.float32, False)):
        if dt == torch.float64:
            Ut, Wt, out = U, W64, out64
        else:
            Ut = [u.to(dt) for u in U]
            Wt = [w.to(dt) for w in W64]
            out = tuple([torch.empty(n, dtype=dt, device=dev) for _ in range(k)] for k in (D * NV, NV * NV, NV))
        per, total = time_launch(lambda: blocks.euler_fused_eos(Ut, Wt, eos, 0, out=out, dw=dw), args.steps,
                                 args.warmup, stream)
        t = max_over_ranks(total / 1e3, world, dev)
        avg = sum(per) / len(per) / 1e3
        b = (PLANES_IN + PLANES_OUT) * BYTES["f32" if dt == torch.float32 else "f64"] * n
        res[tag] = {"value": round(world * n * args.steps / t / 1e9, 3), "unit": UNIT,
                    "ms_per_step": round(t * 1e3 / args.steps, 4), "p99_ms": round(pct(per, 99), 4),
                    "hbm_gbs": round(b / avg / 1e9, 1), "hbm_frac": round(b / avg / 1e9 / hbm_peak, 3),
                    "stated_err": "|gpu - oracle| <= 1e-12 * S" if dt == torch.float64
                    else "|gpu - oracle| <= 2^-24 |o| + 64 * 2^-24 * S"}
        if dt != torch.float64:
            del Ut, Wt, out
    del U
    torch.cuda.empty_cache()
    return res


def time_flushed(fn, steps, warmup, stream, flush):
    """Per-launch CUDA-event times (ms) of fn(); before every timed launch a
    buffer of twice the L2 size is written, so no launch finds its inputs in L2."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        ev = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_configs(args, dev, stream, hbm_peak):
    """The other measurement configurations of the blocks:
    1D N = 65,536 FP64 (19 output planes: V, p, c, w+-, F_x, A_x; L2-resident,
    latency-bound: per-call device time, eager and as one CUDA graph), the
    fused 3D pass swept over N = 2^16 .. 2^24 and at 2^28 (L2 flushed before
    each launch), the precision workload at N = 2^25 (5% near vacuum, 5% at
    Mach 10-50) in every storage form, and the flux VJP at N = 2^24."""
    import torch
    from paper_1809_09851_gb300 import blocks, capi, synth
    L = capi.lib()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    res = {}

    # ---- 1D, N = 65,536 FP64 ------------------------------------------------
    n1 = 65536
    V1 = [torch.from_numpy(v).to(dev) for v in synth.euler1d(n1)]
    U1 = blocks.cons_from_prim(V1, GAMMA)
    # V (3), p, c, w-, w+, F_x (3), A_x (9): 19 planes
    outs = [torch.empty(n1, dtype=torch.float64, device=dev) for _ in range(19)]
    P = lambda ts: capi.planes([t.data_ptr() for t in ts])
    pU, pV, pF, pA = P(U1), P(outs[0:3]), P(outs[7:10]), P(outs[10:19])
    assert len(U1) == 3 and len(outs[10:19]) == 9
    p_, c_, wm, wp = (outs[k].data_ptr() for k in (3, 4, 5, 6))
    calls = {
        "prim_from_cons": lambda st: L.fdbb_prim_from_cons(1, GAMMA, n1, capi.FDBB_F64, pU, pV, st),
        "eos": lambda st: L.fdbb_eos(1, GAMMA, n1, capi.FDBB_F64, pU, p_, c_, st),
        "riemann_inv": lambda st: L.fdbb_riemann_inv(1, 0, GAMMA, n1, capi.FDBB_F64, pU, wm, wp, None, st),
        "flux": lambda st: L.fdbb_flux(1, 0, GAMMA, n1, capi.FDBB_F64, pU, pF, st),
        "flux_jac": lambda st: L.fdbb_flux_jac(1, 0, GAMMA, n1, capi.FDBB_F64, pU, pA, st),
    }
    per_call = {}
    reps = 1000
    with torch.cuda.stream(stream):
        st = stream.cuda_stream
        for name, fn in calls.items():
            for _ in range(10):
                assert fn(st) == 0
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
            torch.cuda.synchronize()
            ev[0].record(stream)
            for i in range(reps):
                fn(st)
                ev[i + 1].record(stream)
            torch.cuda.synchronize()
            t = [ev[i].elapsed_time(ev[i + 1]) * 1e3 for i in range(reps)]
            per_call[name] = {"p50_us": round(pct(t, 50), 2), "p99_us": round(pct(t, 99), 2)}
        # the five calls back to back, eager and replayed as one CUDA graph
        step = lambda st: [fn(st) for fn in calls.values()]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            step(st)
        e1.record(stream)
        torch.cuda.synchronize()
        eager_us = e0.elapsed_time(e1) * 1e3 / reps
    graph_us = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step(torch.cuda.current_stream().cuda_stream)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_us = round(e0.elapsed_time(e1) * 1e3 / reps, 2)
    except Exception as exc:  # capture unsupported: report the eager numbers only
        graph_us = f"unavailable: {type(exc).__name__}"
    res["1d_n65536_f64"] = {"per_call": per_call, "step_eager_us": round(eager_us, 2), "step_graph_us": graph_us,
                            "gpoints_per_s_eager": round(n1 / eager_us / 1e3, 3),
                            "gpoints_per_s_graph": round(n1 / graph_us / 1e3, 3) if isinstance(graph_us, float)
                            else None,
                            "bytes": "24 B in + 152 B out per point; 11.5 MB in all: L2-resident, launch-bound"}
    del V1, U1, outs

    # ---- fused 3D pass, N swept ---------------------------------------------
    sweep = {}
    for lg in (16, 18, 20, 22, 24):
        n = 1 << lg
        U, W = make_fields(n, 1809, dev)
        for tag, dt, dw in (("f64dw", torch.float64, True), ("f32", torch.float32, False)):
            Ut = U if dt == torch.float64 else [u.to(dt) for u in U]
            Wt = W if dt == torch.float64 else [w.to(dt) for w in W]
            out = tuple([torch.empty(n, dtype=dt, device=dev) for _ in range(k)] for k in (D * NV, NV * NV, NV))
            t = time_flushed(lambda: blocks.euler_fused(Ut, Wt, 0, GAMMA, out=out, dw=dw), 20, 3, stream, flush)
            avg = sum(t) / len(t) / 1e3
            b = (PLANES_IN + PLANES_OUT) * (8 if dt == torch.float64 else 4) * n
            sweep[f"2^{lg} {tag}"] = {"gpoints_per_s": round(n / avg / 1e9, 3), "us": round(avg * 1e6, 1),
                                      "hbm_frac": round(b / avg / 1e9 / hbm_peak, 3)}
            del Ut, Wt, out
        del U, W
    torch.cuda.empty_cache()
    # the paper's largest size, N = 2^28 (118 GB of planes in f64): the 2^26
    # field tiled four times on the device
    n = 1 << 28
    U26, W26 = make_fields(1 << 26, 1809, dev)
    U = [u.repeat(4) for u in U26]
    W = [w.repeat(4) for w in W26]
    del U26, W26
    out = tuple([torch.empty(n, dtype=torch.float64, device=dev) for _ in range(k)] for k in (D * NV, NV * NV, NV))
    t = time_flushed(lambda: blocks.euler_fused(U, W, 0, GAMMA, out=out, dw=True), 10, 3, stream, flush)
    avg = sum(t) / len(t) / 1e3
    b = (PLANES_IN + PLANES_OUT) * 8 * n
    sweep["2^28 f64dw"] = {"gpoints_per_s": round(n / avg / 1e9, 3), "us": round(avg * 1e6, 1),
                           "hbm_frac": round(b / avg / 1e9 / hbm_peak, 3), "device_gb": round(b / 1e9, 1)}
    del U, W, out
    torch.cuda.empty_cache()
    res["fused3d_sweep"] = sweep

    # ---- precision workload, N = 2^25 ---------------------------------------
    n = 1 << 25
    case = synth.precision(n)
    V = [torch.from_numpy(v).to(dev) for v in case.V]
    c = blocks.eos(blocks.cons_from_prim(V, GAMMA), GAMMA, want_p=False)[1]  # v = 0 at the fast points
    fast = torch.from_numpy(case.mach > 0).to(dev)
    mach = torch.from_numpy(case.mach).to(dev)
    for k in range(3):
        V[1 + k] = torch.where(fast, mach * c * torch.from_numpy(case.direction[k]).to(dev), V[1 + k])
    U = blocks.cons_from_prim(V, GAMMA)
    W = [torch.from_numpy(w).to(dev) for w in synth.char_weights(n, NV, seed=1810)]
    del V, c, fast, mach, case
    prec = {}
    for tag, dt, dw in (("f64dw", torch.float64, True), ("f32", torch.float32, False),
                        ("f16", torch.float16, False), ("bf16", torch.bfloat16, False)):
        Ut = U if dt == torch.float64 else [u.to(dt) for u in U]
        Wt = W if dt == torch.float64 else [w.to(dt) for w in W]
        out = tuple([torch.empty(n, dtype=dt, device=dev) for _ in range(k)] for k in (D * NV, NV * NV, NV))
        t = time_flushed(lambda: blocks.euler_fused(Ut, Wt, 0, GAMMA, out=out, dw=dw), 20, 3, stream, flush)
        avg = sum(t) / len(t) / 1e3
        b = (PLANES_IN + PLANES_OUT) * torch.empty(0, dtype=dt).element_size() * n
        prec[tag] = {"gpoints_per_s": round(n / avg / 1e9, 3), "hbm_frac": round(b / avg / 1e9 / hbm_peak, 3)}
        del Ut, Wt, out
    prec["workload"] = "2^25 points, 5% near vacuum (rho, p ~ U[1e-4, 1e-3]), 5% at Mach 10-50"
    prec["stated_err"] = "tests/test_gpu_precision.py (arithmetic and end-to-end error per output)"
    res["precision_n2e25"] = prec
    del U, W
    torch.cuda.empty_cache()

    # ---- flux VJP, N = 2^24 --------------------------------------------------
    res["flux_vjp_n2e24"] = run_vjp(1 << 24, dev, stream, hbm_peak, flush)
    del flush
    torch.cuda.empty_cache()
    return res


def run_vjp(n, dev, stream, hbm_peak, flush, steps=20, warmup=3):
    """The flux VJP gU = A_x^T G (10 planes in, 5 out) at N points in FP64
    storage (double-word and IEEE arithmetic) and FP32, L2 flushed before every
    launch."""
    import torch

    from paper_1809_09851_gb300 import blocks, synth

    U, W = make_fields(n, 1809, dev)
    G = [torch.from_numpy(g).to(dev) for g in synth.cotangent(n, NV)]
    vjp = {}
    for tag, dt, dw in (("f64dw", torch.float64, True), ("f64", torch.float64, False), ("f32", torch.float32, False)):
        Ut = U if dt == torch.float64 else [u.to(dt) for u in U]
        Gt = G if dt == torch.float64 else [g.to(dt) for g in G]
        gU = [torch.empty(n, dtype=dt, device=dev) for _ in range(NV)]
        t = time_flushed(lambda: blocks.flux_vjp(Ut, Gt, 0, GAMMA, out=gU, dw=dw), steps, warmup, stream, flush)
        avg = sum(t) / len(t) / 1e3
        b = 15 * (8 if dt == torch.float64 else 4) * n
        vjp[tag] = {"gpoints_per_s": round(n / avg / 1e9, 3), "hbm_frac": round(b / avg / 1e9 / hbm_peak, 3)}
        del Ut, Gt, gU
    del U, W, G
    torch.cuda.empty_cache()
    return vjp


# Building blocks of the per-block leg: name -> (input planes, output planes)
# for the 3D field (U: 5 planes; W / G / U_R: 5 more).
BLOCKS_3D = {
    "v_mag2": (4, 1), "eos": (5, 2), "prim_from_cons": (5, 5), "cons_from_prim": (5, 5),
    "riemann_inv": (5, 2), "flux_x": (5, 5), "flux_all": (5, 15), "flux_jac_x": (5, 25),
    "char_fwd_x": (10, 5), "char_inv_x": (10, 5), "flux_vjp_x": (10, 5), "roe_flux_x": (10, 5),
    "flux_prim_all": (5, 15), "flux_jac_prim_x": (5, 25), "temperature": (5, 1),
}


def run_blocks(n, dev, stream, hbm_peak, steps=10, warmup=3, forms=("f64dw", "f64", "f32", "bf16")):
    """Every building block of the C ABI on its own, 3D, N points: Gpoints/s
    and the fraction of the measured HBM bandwidth its algorithmic bytes (each
    input plane read once, each output plane written once) reach, per storage
    form, timed back to back with CUDA events (every block's planes exceed the
    L2 at N = 2^26, so no flush is needed); and which kernel each launch took."""
    import torch
    from paper_1809_09851_gb300 import blocks, capi
    U64, W64 = make_fields(n, 1809, dev)
    res = {}
    dtypes = {"f64dw": torch.float64, "f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    for form in forms:
        dt = dtypes[form]
        dw = form == "f64dw"
        U = U64 if dt == torch.float64 else [u.to(dt) for u in U64]
        W = W64 if dt == torch.float64 else [w.to(dt) for w in W64]
        V = blocks.prim_from_cons(U, GAMMA, dw=dw)
        UR = [torch.roll(u, 1) for u in U]  # a second physical state for the Roe flux
        out = [torch.empty(n, dtype=dt, device=dev) for _ in range(25)]
        calls = {
            "v_mag2": lambda: blocks.v_mag2(U, out=out[0], dw=dw),
            "eos": lambda: capi.call("fdbb_eos", D, GAMMA, n, blocks._code(dt, dw), blocks._ptrs(U),
                                     out[0].data_ptr(), out[1].data_ptr(), stream.cuda_stream),
            "prim_from_cons": lambda: blocks.prim_from_cons(U, GAMMA, out=out[:5], dw=dw),
            "cons_from_prim": lambda: blocks.cons_from_prim(V, GAMMA, out=out[:5], dw=dw),
            "riemann_inv": lambda: capi.call("fdbb_riemann_inv", D, 0, GAMMA, n, blocks._code(dt, dw),
                                             blocks._ptrs(U), out[0].data_ptr(), out[1].data_ptr(), None,
                                             stream.cuda_stream),
            "flux_x": lambda: blocks.flux(U, 0, GAMMA, out=out[:5], dw=dw),
            "flux_all": lambda: blocks.flux(U, -1, GAMMA, out=out[:15], dw=dw),
            "flux_jac_x": lambda: blocks.flux_jac(U, 0, GAMMA, out=out[:25], dw=dw),
            "char_fwd_x": lambda: blocks.char_transform(U, W, 0, GAMMA, out=out[:5], dw=dw),
            "char_inv_x": lambda: blocks.char_transform(U, W, 0, GAMMA, inverse=True, out=out[:5], dw=dw),
            "flux_vjp_x": lambda: blocks.flux_vjp(U, W, 0, GAMMA, out=out[:5], dw=dw),
            "roe_flux_x": lambda: blocks.roe_flux(U, UR, 0, GAMMA, out=out[:5], dw=dw),
            "flux_prim_all": lambda: blocks.flux_prim(V, -1, GAMMA, out=out[:15], dw=dw),
            "flux_jac_prim_x": lambda: blocks.flux_jac_prim(V, 0, GAMMA, out=out[:25], dw=dw),
            "temperature": lambda: blocks.temperature(U, 2.5, GAMMA, out=out[0], dw=dw),
        }
        es = torch.empty(0, dtype=dt).element_size()
        tab = {}
        for name, fn in calls.items():
            if name not in BLOCKS_3D:
                continue
            pin, pout = BLOCKS_3D[name]
            with torch.cuda.stream(stream):
                fn()
            kind = capi.last_launch().kernel
            per, _ = time_launch(fn, steps, warmup, stream)
            avg = sum(per) / len(per) / 1e3
            gbs = (pin + pout) * es * n / avg / 1e9
            tab[name] = {"gpoints_per_s": round(n / avg / 1e9, 3), "hbm_gbs": round(gbs, 1),
                         "hbm_frac": round(gbs / hbm_peak, 3), "us": round(avg * 1e6, 1),
                         "kernel": {1: "direct", 2: "staged"}.get(kind, "none")}
        tab["bytes_per_point"] = {k: (a + b) * es for k, (a, b) in BLOCKS_3D.items()}
        res[form] = tab
        del U, W, V, UR, out
        torch.cuda.empty_cache()
    res["workload"] = (f"3D field of euler3d_fused, N=2^{int(math.log2(n))}: each block alone (dir 0 where a "
                       "direction applies), every plane read or written once; W doubles as the VJP's G, "
                       "U rolled by one point is the Roe flux's U_R")
    res["note"] = ("f64dw: double-word arithmetic (the inverse characteristic transform runs IEEE double); "
                   "f64: IEEE double, FP64-pipe bound where a block divides or takes square roots")
    del U64, W64
    torch.cuda.empty_cache()
    return res


def pct(xs, q):
    xs = sorted(xs)
    k = max(0, min(len(xs) - 1, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[k]


def run_gpu(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1809_09851_gb300 import blocks, build
    build.build()
    n = args.n
    seed = shard_seed(1809, rank)
    lo = 0
    if args.split and world > 1:
        # strong scaling: the ranks split one n-point field into contiguous ranges
        lo, hi = shard_bounds(args.n, world, rank)
        n, seed = hi - lo, 1809
    stream = torch.cuda.Stream(dev)
    hbm_peak, peak_kind = measured_peaks()
    if args.only == "fv":  # the finite-volume step kernel alone (profiling runs)
        print(json.dumps({"fv_batch": run_fv_batch(args, dev, hbm_peak)}), flush=True)
        return None
    if args.only == "blocks":  # every building block alone at --n points (profiling runs)
        print(json.dumps({"blocks": run_blocks(n, dev, stream, hbm_peak, args.steps, args.warmup,
                                               tuple(args.block_forms.split(",")))}), flush=True)
        return None
    if args.only == "vjp":  # the flux VJP alone at --n points (profiling runs)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"flux_vjp": run_vjp(n, dev, stream, hbm_peak, flush, args.steps, args.warmup)}), flush=True)
        return None

    U64, W64 = make_fields(n, seed, dev, lo)
    alloc = lambda k, dt: [torch.empty(n, dtype=dt, device=dev) for _ in range(k)]
    out64 = (alloc(D * NV, torch.float64), alloc(NV * NV, torch.float64), alloc(NV, torch.float64))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    bytes64 = (PLANES_IN + PLANES_OUT) * BYTES["f64"] * n

    # ---- headline: FP64 storage, double-word arithmetic ------------------------
    # FDBB_F64_DW: every output within 1e-12 of the running-error scale S of
    # the FP64 oracle (the FP64 form's stated error), IEEE double for points
    # outside [2^-24, 2^24]; GB300's FP64 pipe runs at 1/64 of the FP32 rate.
    barrier()
    with ClockSampler(local) as clk:
        per_h, total_h = time_fused(U64, W64, out64, args.steps, args.warmup, stream, dw=True)
    barrier()
    clocks = clk.summary()
    t_max = max_over_ranks(total_h / 1e3, world, dev)
    job_points = args.n if (args.split and world > 1) else world * n  # points of all ranks per step
    value = job_points * args.steps / t_max / 1e9
    avg_h = sum(per_h) / len(per_h) / 1e3
    achieved = bytes64 / avg_h / 1e9
    traffic = recorded_traffic(n)

    # ---- FP64 storage, IEEE double arithmetic ----------------------------------
    f64_native = None
    if args.only in ("all", "f64"):
        barrier()
        per, total = time_fused(U64, W64, out64, args.steps, args.warmup, stream, dw=False)
        barrier()
        t = max_over_ranks(total / 1e3, world, dev)
        avg = sum(per) / len(per) / 1e3
        f64_native = {"value": round(job_points * args.steps / t / 1e9, 3), "unit": UNIT,
                      "ms_per_step": round(t * 1e3 / args.steps, 4),
                      "p50_ms": round(pct(per, 50), 4), "p99_ms": round(pct(per, 99), 4),
                      "hbm_gbs": round(bytes64 / avg / 1e9, 1), "hbm_frac": round(bytes64 / avg / 1e9 / hbm_peak, 3),
                      "bound": "FP64 pipe (2 FP64 ops/clk/SM on GB300; ~70 FP64 ops per point)",
                      "stated_err": "|gpu - oracle| <= 1e-12 * S"}

    # ---- FP32 and BF16 storage (float arithmetic, compensated recovery) -------
    extra = {}
    for tag, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        if args.only not in ("all", tag):
            continue
        U = [u.to(dt) for u in U64]
        W = [w.to(dt) for w in W64]
        out = (alloc(D * NV, dt), alloc(NV * NV, dt), alloc(NV, dt))
        barrier()
        per, total = time_fused(U, W, out, args.steps, args.warmup, stream)
        barrier()
        t = max_over_ranks(total / 1e3, world, dev)
        avg = sum(per) / len(per) / 1e3
        b = (PLANES_IN + PLANES_OUT) * BYTES[tag] * n
        extra[tag] = {"value": round(job_points * args.steps / t / 1e9, 3), "unit": UNIT,
                      "ms_per_step": round(t * 1e3 / args.steps, 4),
                      "p50_ms": round(pct(per, 50), 4), "p99_ms": round(pct(per, 99), 4),
                      "hbm_gbs": round(b / avg / 1e9, 1), "hbm_frac": round(b / avg / 1e9 / hbm_peak, 3),
                      "bytes_per_point": (PLANES_IN + PLANES_OUT) * BYTES[tag]}
        del U, W, out
        torch.cuda.empty_cache()

    # ---- the same pass under a general equation of state -----------------------
    general_eos = None
    if args.only in ("all", "eos"):
        barrier()
        general_eos = run_general_eos(args, n, W64, out64, stream, dev, world, hbm_peak)

    # ---- end to end through host buffers ---------------------------------------
    e2e = None if args.no_e2e else run_e2e(args, U64, W64, out64, stream, dev, world)
    configs = None
    if args.only in ("all", "configs") and world == 1:
        del out64
        torch.cuda.empty_cache()
        out64 = None
        configs = run_configs(args, dev, stream, hbm_peak)
        configs["blocks_n2e26"] = run_blocks(n, dev, stream, hbm_peak)
    del out64
    torch.cuda.empty_cache()
    serving = run_serving(args, dev) if (args.serve_requests > 0 and world == 1) else None
    fv_batch = run_fv_batch(args, dev, hbm_peak) if (args.serve_requests > 0 and world == 1) else None
    if serving is not None:
        serving["fv_step_kernel"] = fv_batch

    result = None
    if rank == 0:
        cpu = cpu_baseline(args) if world == 1 and not args.no_cpu else None
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_max * 1e3 / args.steps, 4),
            "higher_is_better": True, "scaling": "strong" if (args.split and world > 1) else "weak",
            "vs_baseline": None,
            "dtype": "f64 storage, f32x2 double-word arithmetic", "data": "synthetic",
            "stated_err": "|gpu - oracle| <= 1e-12 * S per output (S: running-error scale of the FP64 oracle)",
            "config": {"workload": f"euler3d_fused N=2^{int(math.log2(n))} per GPU, f64 SoA, gamma=1.4, "
                                   "outputs F_x,F_y,F_z + A_x + L_x W",
                       "points_per_gpu": n,
                       "parallelism": (f"dp{world} (one field split into contiguous ranges)"
                                       if (args.split and world > 1) else f"dp{world} (independent fields per GPU)"),
                       "l2": f"inputs+outputs {bytes64 / 1e9:.1f} GB >> L2 {L2_BYTES / 2**20:.0f} MiB: no flush needed"},
            "p50_ms": round(pct(per_h, 50), 4), "p99_ms": round(pct(per_h, 99), 4),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                         "unit": "GB/s", "frac": round(achieved / hbm_peak, 3), "traffic": traffic,
                         "peak_kind": peak_kind, "algorithmic_bytes_per_point": (PLANES_IN + PLANES_OUT) * 8},
            "f64_native": f64_native,
            "mixed": extra,
            "general_eos": general_eos,
            "configs": configs,
            "e2e": e2e,
            "serving": serving,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return result


def run_serving(args, dev):
    """Serving workload: a bounded window of the Poisson request stream
    (2,000 req/s, n^3 periodic grids with n log-uniform in [16, 192], 10-200
    Rusanov steps, FP32 state) through the continuous-batching loop, at the
    full, half and a quarter of the arrival rate; and one-grid-at-a-time FP64
    on a prefix of the same requests."""
    import torch
    from paper_1809_09851_gb300 import serve, synth
    out = {}
    reqs = synth.request_stream(args.serve_requests, rate=2000.0)
    offered = sum(r.n ** 3 * r.steps for r in reqs)
    # the stream's rate, half of it (both above what one GB300 serves, so the
    # latency is mostly queueing) and a quarter (offered below capacity)
    for tag, scale in (("rate_2000", 1.0), ("rate_1000", 2.0), ("rate_500", 4.0)):
        rs = [synth.Request(r.rid, r.arrival * scale, r.n, r.steps, r.seed) for r in reqs]
        srv = serve.FVServer(dev, torch.float32)
        serve.FVServer(dev, torch.float32).run(rs[:4], realtime=False)  # warm-up (kernels, allocator)
        rep = srv.run(rs, realtime=True)
        sm = rep.summary()
        window = rs[-1].arrival
        out[tag] = {"requests": sm["requests"], "p50_s": round(sm["p50_s"], 4), "p99_s": round(sm["p99_s"], 4),
                    "cells_per_s": round(sm["cells_per_s"], 1), "wall_s": round(sm["wall_s"], 3),
                    "offered_cells_per_s": round(offered / window, 1) if window > 0 else None,
                    "max_active": sm["max_active"], "launches": sm["launches"]}
    base = reqs[:args.serve_fp64_requests]
    srv = serve.FVServer(dev, torch.float64, max_active=1)
    rep = srv.run(base, realtime=False)
    sm = rep.summary()
    out["fp64_one_at_a_time"] = {"requests": sm["requests"], "p50_s": round(sm["p50_s"], 4),
                                 "p99_s": round(sm["p99_s"], 4), "cells_per_s": round(sm["cells_per_s"], 1)}
    rep32 = serve.FVServer(dev, torch.float32).run(base, realtime=False)
    out["fp32_batched_same_requests"] = {"cells_per_s": round(rep32.summary()["cells_per_s"], 1)}
    out["workload"] = (f"first {len(reqs)} requests of the Poisson stream (2000/s), n^3 grids n in [16,192] "
                       f"log-uniform, 10-200 steps, CFL 0.4, FP32 state; FP64 baseline on the first {len(base)}")
    return out


def run_fv_batch(args, dev, hbm_peak):
    """Batched Rusanov step kernel alone: 8 periodic 128^3 FP32 grids (16.8 M
    cells) advanced together, 40 B algorithmic traffic per cell-step (5 planes
    read, 5 written)."""
    import torch
    from paper_1809_09851_gb300 import fv
    n, ngrid = args.fv_n, args.fv_grids
    smax = torch.zeros(3 * ngrid, dtype=torch.float32, device=dev)
    grids = [fv.new_grid_smooth(n, 100 + i, i, smax, torch.float32, dev) for i in range(ngrid)]
    for _ in range(max(3, args.warmup)):
        fv.rusanov_step(grids, smax)
    steps = max(3, args.fv_steps)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record()
    for i in range(steps):
        fv.rusanov_step(grids, smax)
        ev[i + 1].record()
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) / 1e3 for i in range(steps)]
    cells = ngrid * n ** 3
    avg = sum(per) / len(per)
    gbs = 40.0 * cells / avg / 1e9
    return {"workload": f"{ngrid} grids of {n}^3, FP32", "cell_steps_per_s": round(cells / avg, 1),
            "ms_per_step": round(avg * 1e3, 4), "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 3),
            "bytes_per_cell_step": 40}


def run_e2e(args, U, W, out, stream, dev, world):
    """Same metric through the public API with pinned host buffers: every step
    moves U and W host->device, runs the fused pass and moves all 45 output
    planes device->host (blocks.euler_fused_host; default mode "mapped_out":
    chunked host->device copies of the inputs overlapped with kernels that
    write their outputs straight into the pinned host planes over the
    CPU-GPU link)."""
    import torch
    from paper_1809_09851_gb300 import blocks
    n = U[0].shape[0]
    steps = max(1, min(args.e2e_steps, args.steps))
    # host fields as single pinned (planes, n) tensors, one row per plane
    hIn = torch.empty(2 * NV, n, dtype=torch.float64, pin_memory=True)
    for k, t in enumerate(list(U) + list(W)):
        hIn[k].copy_(t)
    hOut = torch.empty(PLANES_OUT, n, dtype=torch.float64, pin_memory=True)
    rows_in, rows_out = list(hIn.unbind(0)), list(hOut.unbind(0))
    hU, hW = rows_in[:NV], rows_in[NV:]
    hF, hA, hY = rows_out[:D * NV], rows_out[D * NV:D * NV + NV * NV], rows_out[D * NV + NV * NV:]
    h2d = hIn.numel() * hIn.element_size()
    d2h = hOut.numel() * hOut.element_size()
    with torch.cuda.stream(stream):
        work = blocks.euler_fused_host(hU, hW, (hF, hA, hY), 0, GAMMA, chunk=args.e2e_chunk, device=dev,
                                       dw=True, mode=args.e2e_mode)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            work = blocks.euler_fused_host(hU, hW, (hF, hA, hY), 0, GAMMA, chunk=args.e2e_chunk, device=dev,
                                           work=work, dw=True, mode=args.e2e_mode)
        e1.record(stream)
        torch.cuda.synchronize()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
    del hU, hW, hF, hA, hY, rows_in, rows_out, hIn, hOut, work
    return {"value": round(world * n * steps / t / 1e9, 4), "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": round(t * 1e3 / steps, 3), "mode": args.e2e_mode,
            "chunk_points": args.e2e_chunk if args.e2e_mode != "mapped" else n,
            "gpu_launches_per_step": -(-n // args.e2e_chunk) if args.e2e_mode != "mapped" else 1}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(n_sample, seed=1809):
    import oracle
    from paper_1809_09851_gb300 import synth
    U = oracle.cons_from_prim(D, GAMMA, synth.euler3d(n_sample, seed=seed))
    W = synth.char_weights(n_sample, NV, seed=seed + 1)
    return U, W


def host_cores() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def host_mem_available() -> int:
    """MemAvailable of /proc/meminfo in bytes (0 if unknown)."""
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


class OraclePool:
    """The oracle on all host cores: `cores` threads, each running the unchanged
    FP64 oracle on its contiguous share of the points.  The oracle is a C
    library called through ctypes, which releases the interpreter lock for the
    call, so the threads run in parallel on one shared copy of the inputs.
    run(reps) times every share `reps` times."""

    def __init__(self, U, W, cores=None):
        from concurrent.futures import ThreadPoolExecutor
        self.cores = cores or host_cores()
        ns = U[0].shape[0]
        b = [ns * i // self.cores for i in range(self.cores + 1)]
        self.shares = [([u[b[i]:b[i + 1]] for u in U], [w[b[i]:b[i + 1]] for w in W]) for i in range(self.cores)]
        self.ex = ThreadPoolExecutor(self.cores)
        self.run(1)  # warm: library load, page in

    @staticmethod
    def _share(task):
        import oracle
        (U, W), reps = task
        for _ in range(reps):
            oracle.euler_fused(D, 0, GAMMA, U, W)

    def run(self, reps):
        t0 = time.perf_counter()
        list(self.ex.map(self._share, [(sh, reps) for sh in self.shares]))
        return time.perf_counter() - t0

    def close(self):
        self.ex.shutdown()


def _rates(ns, reps, times):
    """Best and median throughput (Gpoints/s) of timed runs of `reps` passes over `ns` points."""
    r = sorted(ns * reps / t / 1e9 for t in times)
    return round(r[-1], 6), round(r[len(r) // 2], 6)


def _single_runs(U, W, reps, runs):
    """Wall times of `runs` single-thread runs of `reps` oracle passes."""
    import oracle
    oracle.euler_fused(D, 0, GAMMA, U, W)  # warm (load, page in)
    times = []
    for _ in range(runs):
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle.euler_fused(D, 0, GAMMA, U, W)
        times.append(time.perf_counter() - t0)
    return times


def _reps_for(seconds, one_pass):
    return max(1, int(math.ceil(seconds / max(one_pass, 1e-9))))


def cpu_baseline(args):
    """FP64 oracle on the first `cpu_sample` points of the same field, on one
    thread and on all host cores (one thread per core), five timed runs each:
    best and median (the reported value is the all-core median); then the same
    at each size of the sweep (2^16 .. 2^26 points by default, as far as host
    memory allows), every timed run at least `cpu_run_seconds` long.  Every
    size is a prefix of one seeded field (the benchmark's field), generated
    once at the largest size."""
    import oracle
    runs = 5
    cores = getattr(args, "cpu_cores", None) or host_cores()
    sweep_exp = [int(e) for e in str(getattr(args, "cpu_sweep", "16,18,20,22,24,26")).split(",") if e]
    min_run = getattr(args, "cpu_run_seconds", 1.0)
    # each pass holds 10 input and 45 output planes (plus the primitive
    # planes while the field is built): keep it within half of free memory
    avail = host_mem_available()
    fits = lambda m: avail == 0 or 64 * 8 * m <= 0.5 * avail
    sizes = [e for e in sweep_exp if fits(1 << e)]
    skipped = [e for e in sweep_exp if e not in sizes]
    ns = args.cpu_sample
    big = max([ns] + [1 << e for e in sizes])
    U, W = oracle_sample(big)
    pre = lambda m: ([u[:m] for u in U], [w[:m] for w in W])
    Us, Ws = pre(ns)
    oracle.euler_fused(D, 0, GAMMA, Us, Ws)
    t0 = time.perf_counter()
    oracle.euler_fused(D, 0, GAMMA, Us, Ws)
    one = time.perf_counter() - t0
    reps = _reps_for(args.cpu_seconds / runs, one)
    s_best, s_med = _rates(ns, reps, _single_runs(Us, Ws, reps, runs))
    pool = OraclePool(Us, Ws, cores)
    try:
        a_reps = _reps_for(min_run, one / cores)
        a_best, a_med = _rates(ns, a_reps, [pool.run(a_reps) for _ in range(runs)])
    finally:
        pool.close()
    sweep = {}
    for e in sizes:
        m = 1 << e
        Um, Wm = pre(m)
        t0 = time.perf_counter()
        oracle.euler_fused(D, 0, GAMMA, Um, Wm)
        one = time.perf_counter() - t0
        r = _reps_for(min_run, one)
        sb, sm = _rates(m, r, _single_runs(Um, Wm, r, runs))
        p = OraclePool(Um, Wm, cores)
        try:
            ra = _reps_for(min_run, p.run(1))
            ab, am = _rates(m, ra, [p.run(ra) for _ in range(runs)])
        finally:
            p.close()
        sweep[f"2^{e}"] = {"single_best": sb, "single_median": sm, "allcore_best": ab, "allcore_median": am,
                           "passes_per_run": r, "allcore_passes_per_run": ra}
    del U, W
    out = {"value": a_med, "unit": UNIT, "cores": cores, "kind": "oracle",
           "best_value": a_best, "single_thread_value": s_med, "single_thread_best": s_best, "runs": runs,
           "sample": f"first {ns} points of the seeded 3D field, fused pass repeated {reps}x per single-thread "
                     f"run and {a_reps}x per all-core run, {runs} runs on 1 thread and on {cores} threads "
                     f"(one per core; median reported; g++ -O2 -ffp-contract=off)",
           "sweep": sweep, "min_run_s": min_run}
    if skipped:
        out["sweep_skipped"] = {f"2^{e}": "more than half of the host's free memory" for e in skipped}
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    ns = args.ref_sample
    U, W = oracle_sample(ns)
    pool = OraclePool(U, W)
    try:
        for _ in range(args.warmup):
            pool.run(1)
        times = [pool.run(1) for _ in range(args.steps)]
    finally:
        pool.close()
    total = sum(times)
    value = ns * args.steps / total / 1e9
    res = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"euler3d_fused N=2^{int(math.log2(args.n))} per GPU, f64 SoA, gamma=1.4, "
                               "outputs F_x,F_y,F_z + A_x + L_x W",
                   "points_per_gpu": args.n, "parallelism": f"oracle on {pool.cores} host cores"},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": f"each step: first {ns} points of the seeded 3D field split over "
                                   f"{pool.cores} threads, one per core (g++ -O2 -ffp-contract=off)"},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(res), flush=True)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["fdbb", "reference"], default="fdbb")
    ap.add_argument("--n", type=int, default=N_POINTS, help="points per GPU (default 2^26)")
    ap.add_argument("--split", action="store_true",
                    help="with N > 1: split one --n-point field into contiguous ranges (strong scaling) "
                         "instead of one field per rank (weak scaling, the default)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-chunk", type=int, default=1 << 23)
    ap.add_argument("--e2e-mode", choices=["mapped_out", "mapped", "copy"], default="mapped_out",
                    help="how the end-to-end leg moves host data (blocks.euler_fused_host)")
    ap.add_argument("--cpu-sample", type=int, default=1 << 18)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-sweep", default="16,18,20,22,24,26",
                    help="log2 sizes of the oracle sweep (comma-separated; empty: none)")
    ap.add_argument("--cpu-run-seconds", type=float, default=1.0,
                    help="minimum length of each timed oracle run of the sweep")
    ap.add_argument("--ref-sample", type=int, default=1 << 20)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests in the serving window (0 skips the serving leg)")
    ap.add_argument("--serve-fp64-requests", type=int, default=20)
    ap.add_argument("--fv-n", type=int, default=128)
    ap.add_argument("--fv-grids", type=int, default=8)
    ap.add_argument("--fv-steps", type=int, default=20)
    ap.add_argument("--only", choices=["all", "f64", "f32", "bf16", "eos", "configs", "fv", "vjp", "blocks"],
                    default="all", help="storage types to time besides the f64 headline (profiling runs)")
    ap.add_argument("--block-forms", default="f64dw,f64,f32,bf16",
                    help="storage forms of --only blocks (comma-separated)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        print("bench: warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    main()
