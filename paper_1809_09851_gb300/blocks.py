"""Tensor-level wrappers of the C ABI (argument marshalling only).

Fields are lists of 1-D contiguous CUDA tensors, one per component plane, in
the paper's component order (section 2.2): conservative U = (rho, m_1..m_D,
rhoE), primitive V = (rho, v_1..v_D, p).  All planes of a call share one
dtype (float64, float32, float16 or bfloat16) and one length.  Outputs are
allocated with torch unless passed in ``out``; the kernel runs on the current
torch stream (or ``stream``).  Every computation happens in libfdbb.so.

``dw=True`` (float64 planes only) selects double-word arithmetic
(FDBB_F64_DW): the same results to within 1e-12 of each formula's
running-error scale, computed on the float pipe, with IEEE double for points
outside its range.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import capi

DTYPES = {
    torch.float64: capi.FDBB_F64,
    torch.float32: capi.FDBB_F32,
    torch.float16: capi.FDBB_F16,
    torch.bfloat16: capi.FDBB_BF16,
}
GAMMA = 1.4


def check_device() -> None:
    """Synchronise with the device and raise capi.FdbbError (status
    FDBB_ERR_TIMEOUT) if a staged kernel gave up waiting for its input copies
    since the previous check, leaving its outputs unwritten.  Set
    capi.CHECK_DEVICE (or FDBB_CHECK_DEVICE=1) to check after every call."""
    capi.check_device()


def _info(planes: Sequence[torch.Tensor]):
    if not planes:
        raise ValueError("empty field")
    t0 = planes[0]
    for t in planes:
        if not isinstance(t, torch.Tensor):
            raise TypeError("planes must be torch tensors")
        if not t.is_cuda:
            raise ValueError("planes must be CUDA tensors")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError("planes must be contiguous 1-D tensors")
        if t.dtype != t0.dtype or t.shape[0] != t0.shape[0] or t.device != t0.device:
            raise ValueError("planes must share dtype, length and device")
    if t0.dtype not in DTYPES:
        raise TypeError(f"unsupported dtype {t0.dtype}")
    return t0.shape[0], t0.dtype, t0.device


def _code(dtype, dw: bool) -> int:
    if dw:
        if dtype != torch.float64:
            raise TypeError("double-word arithmetic applies to float64 planes only")
        return capi.FDBB_F64_DW
    return DTYPES[dtype]


def _stream(device, stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


def _ptrs(planes):
    return capi.planes([0 if t is None else t.data_ptr() for t in planes])


def _alloc(k, n, dtype, device):
    return [torch.empty(n, dtype=dtype, device=device) for _ in range(k)]


def _dim(U) -> int:
    D = len(U) - 2
    if D not in (1, 2, 3):
        raise ValueError("a field has dim + 2 planes, dim in {1, 2, 3}")
    return D


def v_mag2(U, out: Optional[torch.Tensor] = None, stream=None, dw: bool = False) -> torch.Tensor:
    """|v|^2 = sum m_i^2 / rho^2 (paper section 3, Eq. (2)); U may be nv or D+1 planes."""
    D = len(U) - 2 if len(U) >= 3 else len(U) - 1
    D = min(max(D, 1), 3)
    n, dt, dev = _info(U[: D + 1])
    y = out if out is not None else torch.empty(n, dtype=dt, device=dev)
    capi.call("fdbb_v_mag2", D, n, _code(dt, dw), _ptrs(U[: D + 1]), y.data_ptr(), _stream(dev, stream))
    return y


def prim_from_cons(U, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    n, dt, dev = _info(U)
    V = out if out is not None else _alloc(D + 2, n, dt, dev)
    capi.call("fdbb_prim_from_cons", D, gamma, n, _code(dt, dw), _ptrs(U), _ptrs(V), _stream(dev, stream))
    return V


def cons_from_prim(V, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    D = _dim(V)
    n, dt, dev = _info(V)
    U = out if out is not None else _alloc(D + 2, n, dt, dev)
    capi.call("fdbb_cons_from_prim", D, gamma, n, _code(dt, dw), _ptrs(V), _ptrs(U), _stream(dev, stream))
    return U


def eos(U, gamma: float = GAMMA, want_p: bool = True, want_c: bool = True, stream=None, dw: bool = False):
    """(p, c); an output not wanted is None."""
    D = _dim(U)
    n, dt, dev = _info(U)
    p = torch.empty(n, dtype=dt, device=dev) if want_p else None
    c = torch.empty(n, dtype=dt, device=dev) if want_c else None
    capi.call("fdbb_eos", D, gamma, n, _code(dt, dw), _ptrs(U), p.data_ptr() if p is not None else None,
              c.data_ptr() if c is not None else None, _stream(dev, stream))
    return p, c


def riemann_inv(U, dir: int, gamma: float = GAMMA, entropy: bool = False, stream=None, dw: bool = False):
    """(w-, w+, s) along `dir`; s is None unless entropy=True."""
    D = _dim(U)
    n, dt, dev = _info(U)
    wm, wp = _alloc(2, n, dt, dev)
    s = torch.empty(n, dtype=dt, device=dev) if entropy else None
    capi.call("fdbb_riemann_inv", D, dir, gamma, n, _code(dt, dw), _ptrs(U), wm.data_ptr(), wp.data_ptr(),
              s.data_ptr() if s is not None else None, _stream(dev, stream))
    return wm, wp, s


def flux(U, dir: int = -1, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """F_dir (nv planes) or all directions, direction-major (dim*nv planes)."""
    D = _dim(U)
    n, dt, dev = _info(U)
    k = (D + 2) * (D if dir < 0 else 1)
    F = out if out is not None else _alloc(k, n, dt, dev)
    capi.call("fdbb_flux", D, dir, gamma, n, _code(dt, dw), _ptrs(U), _ptrs(F), _stream(dev, stream))
    return F


def flux_jac(U, dir: int, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """A_dir, nv*nv planes row-major."""
    D = _dim(U)
    n, dt, dev = _info(U)
    A = out if out is not None else _alloc((D + 2) ** 2, n, dt, dev)
    capi.call("fdbb_flux_jac", D, dir, gamma, n, _code(dt, dw), _ptrs(U), _ptrs(A), _stream(dev, stream))
    return A


def char_transform(U, W, dir: int, gamma: float = GAMMA, inverse: bool = False, out=None, stream=None, dw: bool = False):
    """L_dir(U) W, or R_dir(U) W when inverse=True."""
    D = _dim(U)
    n, dt, dev = _info(list(U) + list(W))
    Y = out if out is not None else _alloc(D + 2, n, dt, dev)
    capi.call("fdbb_char_transform", D, dir, gamma, n, _code(dt, dw), int(bool(inverse)), _ptrs(U), _ptrs(W),
              _ptrs(Y), _stream(dev, stream))
    return Y


def euler_fused(U, W, dir_jac: int = 0, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """(F, A, Y): all flux columns, A_dir_jac and L_dir_jac(U) W in one pass.

    ``out`` is an optional (F, A, Y) triple of plane lists (any may be None to
    skip that group); W may be None when Y is skipped.
    """
    D = _dim(U)
    nv = D + 2
    n, dt, dev = _info(list(U) + (list(W) if W is not None else []))
    if out is None:
        out = (_alloc(D * nv, n, dt, dev), _alloc(nv * nv, n, dt, dev),
               _alloc(nv, n, dt, dev) if W is not None else None)
    F, A, Y = out
    capi.call("fdbb_euler_fused", D, dir_jac, gamma, n, _code(dt, dw), _ptrs(U),
              _ptrs(W) if W is not None else None,
              _ptrs(F) if F is not None else None, _ptrs(A) if A is not None else None,
              _ptrs(Y) if Y is not None else None, _stream(dev, stream))
    return F, A, Y


def flux_vjp(U, G, dir: int, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """gU = A_dir(U)^T G."""
    D = _dim(U)
    n, dt, dev = _info(list(U) + list(G))
    gU = out if out is not None else _alloc(D + 2, n, dt, dev)
    capi.call("fdbb_flux_vjp", D, dir, gamma, n, _code(dt, dw), _ptrs(U), _ptrs(G), _ptrs(gU),
              _stream(dev, stream))
    return gU


def flux_prim(V, dir: int = -1, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """Inviscid flux from primitive variables V: F_dir, or all directions for dir == -1."""
    D = _dim(V)
    n, dt, dev = _info(V)
    k = (D + 2) * (D if dir < 0 else 1)
    F = out if out is not None else _alloc(k, n, dt, dev)
    capi.call("fdbb_flux_prim", D, dir, gamma, n, _code(dt, dw), _ptrs(V), _ptrs(F), _stream(dev, stream))
    return F


def flux_jac_prim(V, dir: int, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """dF_dir/dV, nv*nv planes row-major."""
    D = _dim(V)
    n, dt, dev = _info(V)
    B = out if out is not None else _alloc((D + 2) ** 2, n, dt, dev)
    capi.call("fdbb_flux_jac_prim", D, dir, gamma, n, _code(dt, dw), _ptrs(V), _ptrs(B), _stream(dev, stream))
    return B


def temperature(U, cv: float = 2.5, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """T = e / c_v (default c_v = 5/2 of the paper's perfect gas, so T = p / rho)."""
    D = _dim(U)
    n, dt, dev = _info(U)
    T = out if out is not None else torch.empty(n, dtype=dt, device=dev)
    capi.call("fdbb_temperature", D, gamma, cv, n, _code(dt, dw), _ptrs(U), T.data_ptr(), _stream(dev, stream))
    return T


def roe_flux(UL, UR, dir: int, gamma: float = GAMMA, out=None, stream=None, dw: bool = False):
    """Roe flux between the states UL and UR of each point (nv planes)."""
    D = _dim(UL)
    n, dt, dev = _info(list(UL) + list(UR))
    F = out if out is not None else _alloc(D + 2, n, dt, dev)
    capi.call("fdbb_roe_flux", D, dir, gamma, n, _code(dt, dw), _ptrs(UL), _ptrs(UR), _ptrs(F),
              _stream(dev, stream))
    return F


def roe_char_transform(UL, UR, W, dir: int, gamma: float = GAMMA, inverse: bool = False, out=None,
                       stream=None, dw: bool = False):
    """L^ W (or R^ W) at the Roe-averaged state of (UL, UR)."""
    D = _dim(UL)
    n, dt, dev = _info(list(UL) + list(UR) + list(W))
    Y = out if out is not None else _alloc(D + 2, n, dt, dev)
    capi.call("fdbb_roe_char_transform", D, dir, gamma, n, _code(dt, dw), int(bool(inverse)), _ptrs(UL),
              _ptrs(UR), _ptrs(W), _ptrs(Y), _stream(dev, stream))
    return Y


def _info_host(planes: Sequence[torch.Tensor]):
    """Like _info, for planes that are CUDA tensors or pinned CPU tensors."""
    if not planes:
        raise ValueError("empty field")
    t0 = planes[0]
    for t in planes:
        if not isinstance(t, torch.Tensor):
            raise TypeError("planes must be torch tensors")
        if not (t.is_cuda or t.is_pinned()):
            raise ValueError("planes must be CUDA tensors or pinned CPU tensors")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError("planes must be contiguous 1-D tensors")
        if t.dtype != t0.dtype or t.shape[0] != t0.shape[0]:
            raise ValueError("planes must share dtype and length")
    if t0.dtype not in DTYPES:
        raise TypeError(f"unsupported dtype {t0.dtype}")
    return t0.shape[0], t0.dtype


def euler_fused_mapped(U, W, out, dir_jac: int = 0, gamma: float = GAMMA, device=None, stream=None,
                       dw: bool = False):
    """fdbb_euler_fused_host: one launch over planes in pinned host memory
    and/or device memory; the kernel reads and writes host planes directly
    over the CPU-GPU link.  ``out`` is the (F, A, Y) triple of plane lists
    (any may be None); W may be None when Y is None."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    D = _dim(U)
    F, A, Y = out
    n, dt = _info_host(list(U) + (list(W) if W is not None else []) + [p for grp in out if grp for p in grp])
    capi.call("fdbb_euler_fused_host", D, dir_jac, gamma, n, _code(dt, dw), _ptrs(U),
              _ptrs(W) if W is not None else None,
              _ptrs(F) if F is not None else None, _ptrs(A) if A is not None else None,
              _ptrs(Y) if Y is not None else None, _stream(dev, stream))
    return out


def euler_fused_host(U, W, out, dir_jac: int = 0, gamma: float = GAMMA, chunk: int = 1 << 22,
                     device=None, dw: bool = False, work=None, mode: str = "mapped_out"):
    """fdbb_euler_fused over fields in pinned HOST memory.

    U (nv planes) and W (nv planes) are pinned CPU tensors and ``out`` the
    (F, A, Y) plane lists, also pinned CPU tensors (rows of one pinned
    (planes, n) tensor copy fastest).  Modes:

    * ``"mapped_out"`` (default): chunks of ``chunk`` points; the inputs of
      each chunk are copied host-to-device into a device staging buffer (copy
      engine, one stream) while the kernel on the previous chunk, on a second
      stream, reads its staged inputs and writes its outputs straight into the
      host planes over the CPU-GPU link (fdbb_euler_fused_host): the outputs,
      4.5x the inputs' bytes, need no device buffer and no copy.
    * ``"mapped"``: one fdbb_euler_fused_host launch that reads the inputs from
      host memory as well.
    * ``"copy"``: copy engines both ways: host-to-device copy of chunk i+1,
      the kernel on chunk i and the device-to-host copy of chunk i-1 overlap
      on three streams.

    ``work`` may hold the staging buffers of a previous call (returned) to
    avoid reallocating them.  Returns ``work``; the results are complete when
    the current stream has caught up (the call makes the current stream wait
    for its streams).
    """
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if mode == "mapped":
        euler_fused_mapped(U, W, out, dir_jac, gamma, device=dev, dw=dw)
        return work
    if mode not in ("mapped_out", "copy"):
        raise ValueError(f"unknown mode {mode!r}")
    D = _dim(U)
    nv = D + 2
    n = U[0].shape[0]
    dt = U[0].dtype
    F, A, Y = out
    host_out = [*F, *A, *Y]
    n_out = len(host_out)
    nbuf = 2
    copy_out = mode == "copy"
    if work is None or work["chunk"] != chunk or work["dtype"] != dt or work["mode"] != mode:
        work = {
            "chunk": chunk, "dtype": dt, "mode": mode,
            "in": [[torch.empty(chunk, dtype=dt, device=dev) for _ in range(2 * nv)] for _ in range(nbuf)],
            "out": [[torch.empty(chunk, dtype=dt, device=dev) for _ in range(n_out)] for _ in range(nbuf)]
            if copy_out else None,
            "s_h2d": torch.cuda.Stream(dev), "s_cmp": torch.cuda.Stream(dev), "s_d2h": torch.cuda.Stream(dev),
        }
    s_h2d, s_cmp, s_d2h = work["s_h2d"], work["s_cmp"], work["s_d2h"]
    cur = torch.cuda.current_stream(dev)
    for s in (s_h2d, s_cmp, s_d2h):
        s.wait_stream(cur)
    ev_in = [torch.cuda.Event() for _ in range(nbuf)]    # inputs of buffer b staged
    ev_done = [torch.cuda.Event() for _ in range(nbuf)]  # kernel on buffer b finished
    ev_out = [torch.cuda.Event() for _ in range(nbuf)]   # outputs of buffer b copied out
    used = [False] * nbuf
    code = _code(dt, dw)
    nchunks = (n + chunk - 1) // chunk
    for c in range(nchunks):
        b = c % nbuf
        lo, hi = c * chunk, min(n, (c + 1) * chunk)
        m = hi - lo
        din = work["in"][b]
        with torch.cuda.stream(s_h2d):
            if used[b]:
                s_h2d.wait_event(ev_done[b])  # the kernel no longer reads din
            for d, h in zip(din, list(U) + list(W)):
                d[:m].copy_(h[lo:hi], non_blocking=True)
            ev_in[b].record(s_h2d)
        with torch.cuda.stream(s_cmp):
            s_cmp.wait_event(ev_in[b])
            ins = [t[:m] for t in din]
            if copy_out:
                if used[b]:
                    s_cmp.wait_event(ev_out[b])  # dout has been copied out
                outs = [t[:m] for t in work["out"][b]]
            else:
                outs = [h[lo:hi] for h in host_out]
            capi.call("fdbb_euler_fused_host", D, dir_jac, gamma, m, code, _ptrs(ins[:nv]), _ptrs(ins[nv:]),
                      _ptrs(outs[:D * nv]), _ptrs(outs[D * nv:D * nv + nv * nv]), _ptrs(outs[D * nv + nv * nv:]),
                      s_cmp.cuda_stream)
            ev_done[b].record(s_cmp)
        if copy_out:
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(ev_done[b])
                for h, d in zip(host_out, work["out"][b]):
                    h[lo:hi].copy_(d[:m], non_blocking=True)
                ev_out[b].record(s_d2h)
        used[b] = True
    for s in (s_h2d, s_cmp, s_d2h):
        cur.wait_stream(s)
    return work


# ---------------------------------------------------------------------------
# General equations of state (fdbb_*_eos).  ``eos`` is a dict
# {"kind": "ideal" | "nasg" | "vdw", "gamma", "p_inf", "b", "q", "a", "cv"}
# (missing parameters 0, cv 1) or a capi.EosModel.  NASG and VDW take float64
# planes (IEEE double, or double-word with dw=True) or float32 planes;
# "ideal" runs the ideal-gas kernels (any dtype).
# ---------------------------------------------------------------------------

def _eos_ref(eos):
    m = capi.eos_model(eos)
    return m, ctypes.byref(m)


def prim_from_cons_eos(U, eos, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    n, dt, dev = _info(U)
    V = out if out is not None else _alloc(D + 2, n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_prim_from_cons_eos", pm, D, n, _code(dt, dw), _ptrs(U), _ptrs(V), _stream(dev, stream))
    return V


def cons_from_prim_eos(V, eos, out=None, stream=None, dw: bool = False):
    D = _dim(V)
    n, dt, dev = _info(V)
    U = out if out is not None else _alloc(D + 2, n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_cons_from_prim_eos", pm, D, n, _code(dt, dw), _ptrs(V), _ptrs(U), _stream(dev, stream))
    return U


def pressure_eos(U, eos, want_p: bool = True, want_c: bool = True, stream=None, dw: bool = False):
    """(p, c) under the EOS; an output not wanted is None."""
    D = _dim(U)
    n, dt, dev = _info(U)
    p = torch.empty(n, dtype=dt, device=dev) if want_p else None
    c = torch.empty(n, dtype=dt, device=dev) if want_c else None
    m, pm = _eos_ref(eos)
    capi.call("fdbb_pressure_eos", pm, D, n, _code(dt, dw), _ptrs(U), p.data_ptr() if p is not None else None,
              c.data_ptr() if c is not None else None, _stream(dev, stream))
    return p, c


def temperature_eos(U, eos, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    n, dt, dev = _info(U)
    T = out if out is not None else torch.empty(n, dtype=dt, device=dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_temperature_eos", pm, D, n, _code(dt, dw), _ptrs(U), T.data_ptr(), _stream(dev, stream))
    return T


def flux_eos(U, eos, dir: int = -1, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    n, dt, dev = _info(U)
    F = out if out is not None else _alloc((D + 2) * (D if dir < 0 else 1), n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_flux_eos", pm, D, dir, n, _code(dt, dw), _ptrs(U), _ptrs(F), _stream(dev, stream))
    return F


def flux_jac_eos(U, eos, dir: int, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    n, dt, dev = _info(U)
    A = out if out is not None else _alloc((D + 2) ** 2, n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_flux_jac_eos", pm, D, dir, n, _code(dt, dw), _ptrs(U), _ptrs(A), _stream(dev, stream))
    return A


def char_transform_eos(U, W, eos, dir: int, inverse: bool = False, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    n, dt, dev = _info(list(U) + list(W))
    Y = out if out is not None else _alloc(D + 2, n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_char_transform_eos", pm, D, dir, n, _code(dt, dw), int(bool(inverse)), _ptrs(U), _ptrs(W),
              _ptrs(Y), _stream(dev, stream))
    return Y


def euler_fused_eos(U, W, eos, dir_jac: int = 0, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    nv = D + 2
    n, dt, dev = _info(list(U) + (list(W) if W is not None else []))
    if out is None:
        out = (_alloc(D * nv, n, dt, dev), _alloc(nv * nv, n, dt, dev),
               _alloc(nv, n, dt, dev) if W is not None else None)
    F, A, Y = out
    m, pm = _eos_ref(eos)
    capi.call("fdbb_euler_fused_eos", pm, D, dir_jac, n, _code(dt, dw), _ptrs(U),
              _ptrs(W) if W is not None else None,
              _ptrs(F) if F is not None else None, _ptrs(A) if A is not None else None,
              _ptrs(Y) if Y is not None else None, _stream(dev, stream))
    return F, A, Y


def flux_vjp_eos(U, G, eos, dir: int, out=None, stream=None, dw: bool = False):
    D = _dim(U)
    n, dt, dev = _info(list(U) + list(G))
    gU = out if out is not None else _alloc(D + 2, n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_flux_vjp_eos", pm, D, dir, n, _code(dt, dw), _ptrs(U), _ptrs(G), _ptrs(gU), _stream(dev, stream))
    return gU


def flux_prim_eos(V, eos, dir: int = -1, out=None, stream=None, dw: bool = False):
    D = _dim(V)
    n, dt, dev = _info(V)
    F = out if out is not None else _alloc((D + 2) * (D if dir < 0 else 1), n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_flux_prim_eos", pm, D, dir, n, _code(dt, dw), _ptrs(V), _ptrs(F), _stream(dev, stream))
    return F


def flux_jac_prim_eos(V, eos, dir: int, out=None, stream=None, dw: bool = False):
    D = _dim(V)
    n, dt, dev = _info(V)
    B = out if out is not None else _alloc((D + 2) ** 2, n, dt, dev)
    m, pm = _eos_ref(eos)
    capi.call("fdbb_flux_jac_prim_eos", pm, D, dir, n, _code(dt, dw), _ptrs(V), _ptrs(B), _stream(dev, stream))
    return B
