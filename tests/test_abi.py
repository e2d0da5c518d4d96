"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point declared in include/fdbb.h, and rejects bad
arguments before any launch (fake device pointers are never dereferenced
because every call here fails validation or has n == 0)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1809_09851_gb300 import build as lib_build
from paper_1809_09851_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fdbb.h")

A = 1 << 20          # a 16-byte aligned fake address
MIS = (1 << 20) + 8  # an 8-byte (not 16-byte) aligned fake address


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return capi.lib()


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FDBB_API[^;]*?\b(fdbb_[a-z0-9_]+)\s*\(", text, re.S)))


def test_header_declares_the_boundary():
    names = declared()
    for need in ["fdbb_prim_from_cons", "fdbb_cons_from_prim", "fdbb_eos", "fdbb_riemann_inv",
                 "fdbb_flux", "fdbb_flux_jac", "fdbb_char_transform", "fdbb_euler_fused",
                 "fdbb_flux_vjp", "fdbb_v_mag2", "fdbb_status_string"]:
        assert need in names


def test_library_exports_every_declared_symbol(L):
    for name in declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_build.LIBRARY], capture_output=True, text=True)
    exported = set(re.findall(r"\sT\s(\w+)", out.stdout))
    assert set(declared()) <= exported
    # nothing but the C ABI leaks out of the shared object
    assert all(s.startswith("fdbb_") or s.startswith("_") for s in exported), sorted(exported)[:10]


def test_status_strings(L):
    assert capi.status_string(0) == "ok"
    assert "aligned" in capi.status_string(3)
    assert L.fdbb_version() >= 100


def _U(k, addr=A):
    return capi.planes([addr + 256 * i for i in range(k)])


def test_argument_errors_return_before_launch(L):
    F64 = capi.FDBB_F64
    # dim out of range
    assert L.fdbb_flux(4, 0, 1.4, 10, F64, _U(6), _U(6), None) == 1
    # dir out of range
    assert L.fdbb_flux(3, 3, 1.4, 10, F64, _U(5), _U(5), None) == 1
    assert L.fdbb_flux_jac(2, -1, 1.4, 10, F64, _U(4), _U(16), None) == 1
    # gamma <= 1
    assert L.fdbb_eos(3, 1.0, 10, F64, _U(5), A, A, None) == 1
    # n < 0
    assert L.fdbb_prim_from_cons(3, 1.4, -1, F64, _U(5), _U(5), None) == 1
    # NULL input array / NULL input plane
    assert L.fdbb_flux(3, 0, 1.4, 10, F64, None, _U(5), None) == 2
    assert L.fdbb_flux(3, 0, 1.4, 10, F64, capi.planes([A, 0, A, A, A]), _U(5), None) == 2
    # misaligned input / output plane
    assert L.fdbb_flux(3, 0, 1.4, 10, F64, _U(5, MIS), _U(5), None) == 3
    assert L.fdbb_flux_jac(3, 0, 1.4, 10, F64, _U(5), capi.planes([A] * 24 + [MIS]), None) == 3
    # unknown storage type
    assert L.fdbb_flux(3, 0, 1.4, 10, 9, _U(5), _U(5), None) == 4
    # fused: W required when Y is wanted
    assert L.fdbb_euler_fused(3, 0, 1.4, 10, F64, _U(5), None, None, None, _U(5), None) == 2


def test_empty_input_is_a_no_op(L):
    # n == 0 validates the arguments and returns without touching the device
    assert L.fdbb_flux(3, -1, 1.4, 0, capi.FDBB_F32, _U(5), _U(15), None) == 0
    assert L.fdbb_euler_fused(3, 0, 1.4, 0, capi.FDBB_F64, _U(5), _U(5), _U(15), _U(25), _U(5), None) == 0


def _eos(**kw):
    d = {"kind": "nasg", "gamma": 1.6, "p_inf": 1.0, "b": 0.1, "q": -0.3, "cv": 2.0}
    d.update(kw)
    return ctypes.byref(capi.eos_model(d))


def test_general_eos_argument_errors(L):
    F64, F32 = capi.FDBB_F64, capi.FDBB_F32
    # NULL model, bad parameters, reserved field
    assert L.fdbb_flux_eos(None, 3, 0, 10, F64, _U(5), _U(5), None) == 1
    for bad in ({"gamma": 1.0}, {"cv": 0.0}, {"b": -0.1}, {"p_inf": -1.0}, {"kind": "vdw", "a": -1.0}):
        assert L.fdbb_pressure_eos(_eos(**bad), 3, 10, F64, _U(5), A, A, None) == 1, bad
    m = capi.eos_model({"kind": "nasg", "gamma": 1.4})
    m.reserved = 1
    assert L.fdbb_flux_eos(ctypes.byref(m), 3, 0, 10, F64, _U(5), _U(5), None) == 1
    m = capi.eos_model({"kind": "nasg", "gamma": 1.4})
    m.kind = 7
    assert L.fdbb_flux_eos(ctypes.byref(m), 3, 0, 10, F64, _U(5), _U(5), None) == 1
    # dim / dir / n
    assert L.fdbb_flux_eos(_eos(), 4, 0, 10, F64, _U(6), _U(6), None) == 1
    assert L.fdbb_flux_jac_eos(_eos(), 2, -1, 10, F64, _U(4), _U(16), None) == 1
    assert L.fdbb_prim_from_cons_eos(_eos(), 3, -1, F64, _U(5), _U(5), None) == 1
    # an unknown storage type
    assert L.fdbb_flux_eos(_eos(), 3, 0, 10, 9, _U(5), _U(5), None) == 4
    # NULL / misaligned planes, W required for Y in the fused pass
    assert L.fdbb_flux_eos(_eos(), 3, 0, 10, F32, None, _U(5), None) == 2
    assert L.fdbb_temperature_eos(_eos(), 3, 10, F64, _U(5), None, None) == 2
    assert L.fdbb_flux_vjp_eos(_eos(), 3, 0, 10, F64, _U(5, MIS), _U(5), _U(5), None) == 3
    assert L.fdbb_euler_fused_eos(_eos(), 3, 0, 10, F64, _U(5), None, None, None, _U(5), None) == 2
    # the ideal kind forwards to the ideal-gas entry points and their checks
    ideal = _eos(kind="ideal", gamma=1.4)
    assert L.fdbb_flux_eos(ideal, 3, 3, 10, F64, _U(5), _U(5), None) == 1
    assert L.fdbb_flux_eos(ideal, 3, 0, 10, capi.FDBB_BF16, _U(5, MIS), _U(5), None) == 3


def test_general_eos_empty_input_is_a_no_op(L):
    for kind in ("nasg", "vdw", "ideal"):
        m = _eos(kind=kind, a=0.05)
        assert L.fdbb_euler_fused_eos(m, 3, 1, 0, capi.FDBB_F64, _U(5), _U(5), _U(15), _U(25), _U(5), None) == 0
        assert L.fdbb_cons_from_prim_eos(m, 2, 0, capi.FDBB_F32, _U(4), _U(4), None) == 0
        assert L.fdbb_flux_jac_prim_eos(m, 1, 0, 0, capi.FDBB_F64, _U(3), _U(9), None) == 0


def test_pointer_kind_of_host_memory(L):
    """NULL and pageable host memory are never plane memory the device can use
    (on a machine without a GPU every query answers FDBB_PTR_OTHER)."""
    buf = ctypes.create_string_buffer(64)
    assert L.fdbb_pointer_kind(None) == capi.FDBB_PTR_OTHER
    assert L.fdbb_pointer_kind(ctypes.addressof(buf)) == capi.FDBB_PTR_OTHER


def test_fv_init_smooth_argument_errors(L):
    g = capi.FvGrid()
    for q in range(5):
        g.U[q] = A + 256 * q
    g.n = 8
    wave = (ctypes.c_double * 30)(*([1.0] * 30))
    F32, F64 = capi.FDBB_F32, capi.FDBB_F64
    assert L.fdbb_fv_init_smooth(None, 1.4, 0.1, wave, F32, A, None) == 2
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, None, F32, A, None) == 2
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, wave, F32, None, None) == 2
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, wave, capi.FDBB_BF16, A, None) == 4
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.0, 0.1, wave, F32, A, None) == 1
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, float("nan"), wave, F32, A, None) == 1
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, wave, F64, A + 4, None) == 3
    g.n = 0
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, wave, F32, A, None) == 1
    g.n = 8
    g.U[3] = None
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, wave, F32, A, None) == 2
    g.U[3] = MIS
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, wave, F32, A, None) == 3
    bad = (ctypes.c_double * 30)(*([1.0] * 29 + [float("inf")]))
    g.U[3] = A + 768
    assert L.fdbb_fv_init_smooth(ctypes.byref(g), 1.4, 0.1, bad, F32, A, None) == 1


def test_launch_record_and_wait_limit_need_no_device(L):
    """fdbb_last_launch and fdbb_set_wait_limit are host-side: a thread that
    launched nothing reports FDBB_KERNEL_NONE, NULL is rejected, and the wait
    limit setting round-trips (negative values restore the default, -1)."""
    import threading
    out = {}

    def probe():
        out["info"] = capi.last_launch()

    t = threading.Thread(target=probe)
    t.start()
    t.join()
    assert out["info"].kernel == capi.FDBB_KERNEL_NONE
    assert L.fdbb_last_launch(None) == 2
    prev = L.fdbb_set_wait_limit(5)
    try:
        assert L.fdbb_set_wait_limit(0) == 5
        assert L.fdbb_set_wait_limit(-7) == 0
        assert L.fdbb_set_wait_limit(-1) == -1
    finally:
        L.fdbb_set_wait_limit(prev)


def test_release_build_has_no_index_checks(L):
    """The release library compiles the kernels' index checks out: the debug
    query answers -1 without touching the device."""
    assert capi.debug_index_faults() == (-1, -1)
