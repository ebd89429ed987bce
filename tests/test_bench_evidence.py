"""The benchmark's link to its ncu evidence (CPU): the DRAM traffic of the
committed capture is reported only while the library's CUDA sources (kernels
and the host code that lays out their scratch and sizes their grids), the
header's constants and the nvcc flags are the ones it was taken on.  Header
comments do not enter the hash."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_tree(tmp_path, monkeypatch):
    """A copy of the sources and profiles whose capture is marked as taken on
    the copied kernel sources."""
    for d in ("paper_2412_14966_gb300/csrc", "include", "profiles"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(tmp_path, d))
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    prof = os.path.join(root, "profiles", "fused_kernel_nominal.md")
    lines = [ln for ln in open(prof).read().splitlines() if not ln.startswith("sources_hash:")]
    with open(prof, "w") as f:
        f.write("\n".join(lines + [f"sources_hash: {bench._sources_hash()}", ""]))
    return root


def _append(path, text):
    with open(path, "a") as f:
        f.write(text)


def test_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path, monkeypatch)
    h0 = bench._sources_hash()
    traffic = bench._profiled_traffic(10_000)
    assert traffic is not None and traffic > 0
    # header comments do not invalidate it
    _append(os.path.join(root, "include", "pv.h"), "\n/* a comment */\n")
    assert bench._sources_hash() == h0
    assert bench._profiled_traffic(10_000) == traffic
    # a header constant does
    _append(os.path.join(root, "include", "pv.h"), "#define PV_SOMETHING 1\n")
    h1 = bench._sources_hash()
    assert h1 != h0 and bench._profiled_traffic(10_000) is None


def test_traffic_is_dropped_when_the_build_flags_change(tmp_path, monkeypatch):
    _copy_tree(tmp_path, monkeypatch)
    from paper_2412_14966_gb300 import build
    h0 = bench._sources_hash()
    monkeypatch.setattr(build, "NVCC_FLAGS", build.NVCC_FLAGS + ["-DSOMETHING"])
    assert bench._sources_hash() != h0
    assert bench._profiled_traffic(10_000) is None


def test_traffic_is_dropped_when_a_kernel_changes(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path, monkeypatch)
    h0 = bench._sources_hash()
    assert bench._profiled_traffic(10_000) is not None
    for f in ("pv_device.cuh", "pv_kernels.cu", "pv_kernels.cuh", "pv_api.cu"):
        p = os.path.join(root, "paper_2412_14966_gb300", "csrc", f)
        saved = open(p).read()
        _append(p, "\n// changed\n")
        assert bench._sources_hash() != h0, f
        assert bench._profiled_traffic(10_000) is None, f
        with open(p, "w") as fh:
            fh.write(saved)
    assert bench._sources_hash() == h0
