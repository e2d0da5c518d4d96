"""ctypes binding of the C ABI in include/fdbb.h (argument marshalling only).

``lib()`` loads ``libfdbb.so`` from the package directory (with the
environment variable FDBB_DEBUG=1: ``libfdbb_debug.so``, the build whose
kernels check every index, see ``fdbb_debug_index_faults``).  There is no
fallback: if the library has not been built (``paper_1809_09851_gb300.build``)
every call raises.  The raw functions keep the C names (``fdbb_flux`` ...) and
take plane-pointer arrays built with :func:`planes`.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIBRARY, LIBRARY_DEBUG

if os.environ.get("FDBB_DEBUG", "0") == "1":
    LIBRARY = LIBRARY_DEBUG  # noqa: F811 - the debug build replaces the release one

FDBB_OK = 0
STATUS = {
    0: "FDBB_OK", 1: "FDBB_ERR_ARG", 2: "FDBB_ERR_NULLPTR", 3: "FDBB_ERR_ALIGN",
    4: "FDBB_ERR_DTYPE", 5: "FDBB_ERR_CUDA", 6: "FDBB_ERR_TIMEOUT", 7: "FDBB_ERR_NOMEM",
}
STATUS_CODES = {name: code for code, name in STATUS.items()}
FDBB_F64, FDBB_F32, FDBB_F16, FDBB_BF16, FDBB_F64_DW = 0, 1, 2, 3, 4
FDBB_PTR_OTHER, FDBB_PTR_DEVICE, FDBB_PTR_HOST, FDBB_PTR_MANAGED = 0, 1, 2, 3

_i, _i64, _d, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)

# name -> argument types (the return type is int status unless noted)
SIGNATURES = {
    "fdbb_v_mag2": [_i, _i64, _i, _PP, _vp, _vp],
    "fdbb_prim_from_cons": [_i, _d, _i64, _i, _PP, _PP, _vp],
    "fdbb_cons_from_prim": [_i, _d, _i64, _i, _PP, _PP, _vp],
    "fdbb_eos": [_i, _d, _i64, _i, _PP, _vp, _vp, _vp],
    "fdbb_riemann_inv": [_i, _i, _d, _i64, _i, _PP, _vp, _vp, _vp, _vp],
    "fdbb_flux": [_i, _i, _d, _i64, _i, _PP, _PP, _vp],
    "fdbb_flux_jac": [_i, _i, _d, _i64, _i, _PP, _PP, _vp],
    "fdbb_char_transform": [_i, _i, _d, _i64, _i, _i, _PP, _PP, _PP, _vp],
    "fdbb_euler_fused": [_i, _i, _d, _i64, _i, _PP, _PP, _PP, _PP, _PP, _vp],
    "fdbb_euler_fused_host": [_i, _i, _d, _i64, _i, _PP, _PP, _PP, _PP, _PP, _vp],
    "fdbb_flux_vjp": [_i, _i, _d, _i64, _i, _PP, _PP, _PP, _vp],
    "fdbb_roe_flux": [_i, _i, _d, _i64, _i, _PP, _PP, _PP, _vp],
    "fdbb_flux_prim": [_i, _i, _d, _i64, _i, _PP, _PP, _vp],
    "fdbb_flux_jac_prim": [_i, _i, _d, _i64, _i, _PP, _PP, _vp],
    "fdbb_temperature": [_i, _d, _d, _i64, _i, _PP, _vp, _vp],
    "fdbb_roe_char_transform": [_i, _i, _d, _i64, _i, _i, _PP, _PP, _PP, _PP, _vp],
}



class FvGrid(ctypes.Structure):
    """struct fdbb_fv_grid (include/fdbb.h)."""
    _fields_ = [("U", ctypes.c_void_p * 5), ("Unew", ctypes.c_void_p * 5), ("dt_log", ctypes.c_void_p),
                ("cell_begin", ctypes.c_int64), ("n", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("phase", ctypes.c_int32), ("step", ctypes.c_int32)]


FV_TILE = 256
FV_MAX_GRIDS = 256
_FVP = ctypes.POINTER(FvGrid)
SIGNATURES.update({
    "fdbb_fv_max_speed": [_i, _FVP, _i64, _d, _i, _vp, _vp],
    "fdbb_fv_rusanov_step": [_i, _FVP, _i64, _d, _d, _i, _vp, _vp],
    "fdbb_fv_rusanov_step_noalloc": [_i, _FVP, _i64, _d, _d, _i, _vp],
    "fdbb_fv_init_smooth": [_FVP, _d, _d, _vp, _i, _vp, _vp],
})



class EosModel(ctypes.Structure):
    """struct fdbb_eos_model (include/fdbb.h)."""
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("p_inf", ctypes.c_double), ("b", ctypes.c_double), ("q", ctypes.c_double),
                ("a", ctypes.c_double), ("cv", ctypes.c_double)]


FDBB_EOS_IDEAL, FDBB_EOS_NASG, FDBB_EOS_VDW = 0, 1, 2
EOS_KINDS = {"ideal": FDBB_EOS_IDEAL, "nasg": FDBB_EOS_NASG, "vdw": FDBB_EOS_VDW}


def eos_model(eos) -> EosModel:
    """EosModel from a dict {"kind": "ideal"|"nasg"|"vdw", "gamma", "p_inf", "b",
    "q", "a", "cv"} (missing parameters 0, cv 1) or an EosModel."""
    if isinstance(eos, EosModel):
        return eos
    return EosModel(EOS_KINDS[eos["kind"]], 0, float(eos["gamma"]), float(eos.get("p_inf", 0.0)),
                    float(eos.get("b", 0.0)), float(eos.get("q", 0.0)), float(eos.get("a", 0.0)),
                    float(eos.get("cv", 1.0)))


_EP = ctypes.POINTER(EosModel)
SIGNATURES.update({
    "fdbb_prim_from_cons_eos": [_EP, _i, _i64, _i, _PP, _PP, _vp],
    "fdbb_cons_from_prim_eos": [_EP, _i, _i64, _i, _PP, _PP, _vp],
    "fdbb_pressure_eos": [_EP, _i, _i64, _i, _PP, _vp, _vp, _vp],
    "fdbb_temperature_eos": [_EP, _i, _i64, _i, _PP, _vp, _vp],
    "fdbb_flux_eos": [_EP, _i, _i, _i64, _i, _PP, _PP, _vp],
    "fdbb_flux_jac_eos": [_EP, _i, _i, _i64, _i, _PP, _PP, _vp],
    "fdbb_char_transform_eos": [_EP, _i, _i, _i64, _i, _i, _PP, _PP, _PP, _vp],
    "fdbb_euler_fused_eos": [_EP, _i, _i, _i64, _i, _PP, _PP, _PP, _PP, _PP, _vp],
    "fdbb_flux_vjp_eos": [_EP, _i, _i, _i64, _i, _PP, _PP, _PP, _vp],
    "fdbb_flux_prim_eos": [_EP, _i, _i, _i64, _i, _PP, _PP, _vp],
    "fdbb_flux_jac_prim_eos": [_EP, _i, _i, _i64, _i, _PP, _PP, _vp],
})

class LaunchInfo(ctypes.Structure):
    """struct fdbb_launch_info (include/fdbb.h)."""
    _fields_ = [("kernel", ctypes.c_int32), ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("points_per_thread", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


FDBB_KERNEL_NONE, FDBB_KERNEL_DIRECT, FDBB_KERNEL_STAGED = 0, 1, 2
SIGNATURES["fdbb_last_launch"] = [ctypes.POINTER(LaunchInfo)]

_lib = None


class FdbbError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} returned {STATUS.get(status, status)}")
        self.status = status


def lib():
    """Load libfdbb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBRARY):
            raise RuntimeError(
                f"{LIBRARY} is missing: build the CUDA library first "
                "(python -m paper_1809_09851_gb300.build or __graft_entry__.build())")
        L = ctypes.CDLL(LIBRARY)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _i
        L.fdbb_status_string.argtypes = [_i]
        L.fdbb_status_string.restype = ctypes.c_char_p
        L.fdbb_version.argtypes = []
        L.fdbb_version.restype = _i
        L.fdbb_device_status.argtypes = []
        L.fdbb_device_status.restype = _i
        L.fdbb_pointer_kind.argtypes = [_vp]
        L.fdbb_pointer_kind.restype = _i
        L.fdbb_set_wait_limit.argtypes = [_i]
        L.fdbb_set_wait_limit.restype = _i
        L.fdbb_debug_index_faults.argtypes = [ctypes.POINTER(ctypes.c_int64)]
        L.fdbb_debug_index_faults.restype = ctypes.c_int64
        _lib = L
    return _lib


def planes(ptrs):
    """Host array of device plane pointers (ints or None) for a C call."""
    if ptrs is None:
        return None
    return (ctypes.c_void_p * max(1, len(ptrs)))(*[p if p else None for p in ptrs])


# With CHECK_DEVICE (environment FDBB_CHECK_DEVICE=1) every launching call
# synchronises with the device afterwards and raises FdbbError(FDBB_ERR_TIMEOUT)
# if a staged kernel's bounded wait for its input copies ran out (that kernel
# left its outputs unwritten).  Off by default: it makes every call blocking.
CHECK_DEVICE = os.environ.get("FDBB_CHECK_DEVICE", "0") == "1"
_NO_LAUNCH = {"fdbb_last_launch"}


def check_device() -> None:
    """Synchronise and raise FdbbError if a bounded device wait ran out since
    the previous check (fdbb_device_status)."""
    st = device_status()
    if st != FDBB_OK:
        raise FdbbError("fdbb_device_status", st)


def call(name: str, *args) -> None:
    """Call fdbb_<name> and raise FdbbError on a non-zero status."""
    st = getattr(lib(), name)(*args)
    if st != FDBB_OK:
        raise FdbbError(name, st)
    if CHECK_DEVICE and name not in _NO_LAUNCH:
        check_device()


def last_launch() -> LaunchInfo:
    """Kernel, grid and shared memory of this thread's last point-wise launch."""
    info = LaunchInfo()
    call("fdbb_last_launch", ctypes.byref(info))
    return info


def device_status() -> int:
    """fdbb_device_status(): synchronises; FDBB_ERR_TIMEOUT if a bounded device
    wait ran out since the previous call, else FDBB_OK."""
    return lib().fdbb_device_status()


def debug_index_faults():
    """(violations since the last call, first offending index) of a debug
    build's kernel index checks; (-1, -1) for a release build."""
    first = ctypes.c_int64(-1)
    count = lib().fdbb_debug_index_faults(ctypes.byref(first))
    return int(count), int(first.value)


def status_string(status: int) -> str:
    return lib().fdbb_status_string(status).decode()


def exported_symbols():
    return ["fdbb_status_string", "fdbb_version", "fdbb_device_status", "fdbb_pointer_kind", "fdbb_set_wait_limit",
            "fdbb_debug_index_faults", *SIGNATURES.keys()]
