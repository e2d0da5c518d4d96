"""Host-side bookkeeping of the benchmark (no GPU): the recorded ncu traffic
of the headline kernel is reported only for the kernel sources it was taken
on."""
import os
import shutil

import bench


def _copy_sources(dst):
    src_dir = os.path.join(bench.ROOT, "paper_1809_09851_gb300", "csrc")
    dst_dir = os.path.join(dst, "paper_1809_09851_gb300", "csrc")
    os.makedirs(dst_dir)
    for f in bench.FUSED_KERNEL_SOURCES:
        shutil.copy(os.path.join(src_dir, f), dst_dir)
    return dst_dir


def test_source_hash_follows_every_byte(tmp_path):
    d = _copy_sources(str(tmp_path))
    h0 = bench.kernel_source_hash(str(tmp_path))
    assert h0 == bench.kernel_source_hash()
    for f in bench.FUSED_KERNEL_SOURCES:
        p = os.path.join(d, f)
        body = open(p, "rb").read()
        open(p, "wb").write(body + b"\n")
        assert bench.kernel_source_hash(str(tmp_path)) != h0, f
        open(p, "wb").write(body)
    assert bench.kernel_source_hash(str(tmp_path)) == h0


def test_traffic_only_for_the_recorded_sources(tmp_path, monkeypatch):
    d = _copy_sources(str(tmp_path))
    h = bench.kernel_source_hash(str(tmp_path))
    monkeypatch.setitem(bench.NCU_TRAFFIC, "source_hash", h)
    monkeypatch.setitem(bench.NCU_TRAFFIC, "bytes_per_point", 425.0)
    assert bench.recorded_traffic(1 << 26, str(tmp_path)) == round(425.0 * (1 << 26))
    with open(os.path.join(d, "fdbb_kernels.cuh"), "ab") as fh:
        fh.write(b"// changed\n")
    assert bench.recorded_traffic(1 << 26, str(tmp_path)) is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "bytes_per_point", None)
    assert bench.recorded_traffic(1 << 26) is None
