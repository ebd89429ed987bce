"""The C ABI library builds for sm_103a, loads, and exports every function
include/pv.h declares; the ctypes layouts match the C structs.  CPU only: no
kernel is launched."""
import ctypes
import json
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pv.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2412_14966_gb300 import build
    build.build()
    import paper_2412_14966_gb300 as pv
    return pv.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pv_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    import paper_2412_14966_gb300 as pv
    assert sorted(pv.EXPORTED) == names


def test_library_is_built_for_sm_103a():
    from paper_2412_14966_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True)
    for n in declared_functions():
        assert re.search(rf"\bT {n}\b", out.stdout), n


def _c_layout():
    """sizeof / offsetof of the ABI structs as the C compiler sees them."""
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "pv.h"
#define F(T, m) printf("\"" #T "." #m "\": %zu,\n", offsetof(T, m))
int main(void) {
  printf("{\n");
  F(pv_config, z_min); F(pv_config, bin_threshold); F(pv_config, chi2_max);
  F(pv_config, max_iter); F(pv_config, accum_mode); F(pv_config, path);
  F(pv_config, pool_bytes); F(pv_config, max_spin_ns); F(pv_config, mv_chi2_cut);
  F(pv_config, mv_dup_sep2);
  F(pv_tracks, x); F(pv_tracks, ctyty); F(pv_tracks, event_offsets);
  F(pv_tracks, n_tracks); F(pv_tracks, n_events);
  F(pv_vertices, x); F(pv_vertices, cov); F(pv_vertices, bin_max);
  F(pv_vertices, n_per_event); F(pv_vertices, track_vertex); F(pv_vertices, capacity);
  printf("\"sizeof.pv_config\": %zu, \"sizeof.pv_tracks\": %zu, \"sizeof.pv_vertices\": %zu,"
         " \"sizeof.pv_beamline\": %zu}\n", sizeof(pv_config), sizeof(pv_tracks),
         sizeof(pv_vertices), sizeof(pv_beamline));
  return 0;
}
"""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "l")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        return json.loads(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)


def test_ctypes_layout_matches_c(lib):
    import paper_2412_14966_gb300 as pv
    lay = _c_layout()
    for name, cls in (("pv_config", pv.pv_config), ("pv_tracks", pv.pv_tracks),
                      ("pv_vertices", pv.pv_vertices), ("pv_beamline", pv.pv_beamline)):
        assert ctypes.sizeof(cls) == lay[f"sizeof.{name}"], name
    for key, off in lay.items():
        if key.startswith("sizeof."):
            continue
        struct, field = key.split(".")
        cls = getattr(pv, struct)
        assert getattr(cls, field).offset == off, key


def test_default_config_is_the_papers(lib):
    """pv_config_default holds the paper's constants (same golden file as the
    oracle's defaults)."""
    import paper_2412_14966_gb300 as pv
    import oracle
    with open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")) as f:
        g = json.load(f)
    c = pv.default_config()
    assert c.z_min == g["histogram_z_min_mm"]["value"]
    assert c.z_max == g["histogram_z_max_mm"]["value"]
    assert c.dz == g["bin_width_mm"]["value"]
    assert abs(c.sigma_max_pp - g["sigma_max_pp_mm"]["value"]) < 1e-6
    assert c.sigma_max_gas == g["sigma_max_gas_mm"]["value"]
    assert c.z_gas == g["gas_region_upper_z_mm"]["value"]
    assert c.min_integral_pp == g["min_cluster_integral_pp"]["value"]
    assert c.min_integral_gas == g["min_cluster_integral_gas"]["value"]
    assert c.min_pv_tracks_pp == g["min_tracks_pv_pp"]["value"]
    assert c.min_pv_tracks_gas == g["min_tracks_pv_gas"]["value"]
    assert c.min_assoc_pp == g["min_assoc_tracks_pp"]["value"]
    assert c.min_assoc_gas == g["min_assoc_tracks_gas"]["value"]
    assert c.chi2_max == g["tukey_chi2_max"]["value"]
    assert abs(c.dchi2_tol - g["converge_dchi2"]["value"]) < 1e-9
    assert abs(c.dz_tol - g["converge_dz_mm"]["value"]) < 1e-9
    assert c.max_iter == g["max_iterations"]["value"]
    assert abs(c.max_r_beam - g["max_beamline_distance_mm"]["value"]) < 1e-7
    assert c.mv_chi2_cut == g["multivertex_chi2_max"]["value"]
    assert abs(c.mv_dz_tol - g["gpu_converge_dz_mm"]["value"]) < 1e-9
    assert c.mv_dup_sep2 == g["duplicate_separation"]["value"]
    m = oracle.default_mv_params()
    assert (m.chi2_cut, m.dup_sep2, m.w_assoc) == (c.mv_chi2_cut, c.mv_dup_sep2, c.mv_w_assoc)
    assert abs(m.dz_tol - c.mv_dz_tol) < 1e-9
    # the unstated settings agree between library and oracle
    p = oracle.default_params()
    assert (c.bin_threshold, c.dip_num, c.dip_den) == (p.bin_threshold, p.dip_num, p.dip_den)
    assert c.split_mode == p.split_mode == pv.SPLIT_ZORDER
    assert c.profile_mode == p.profile_mode == pv.PROFILE_CUBIC


@pytest.mark.parametrize("field,value", [("split_mode", 2), ("split_mode", -1),
                                         ("profile_mode", 2), ("dz", 0.0), ("mv_chi2_cut", 0.0)])
def test_invalid_config_is_refused_before_the_device(lib, field, value):
    """pv_init checks the configuration before it looks for a device."""
    import paper_2412_14966_gb300 as pv
    cfg = pv.default_config(**{field: value})
    beam = pv.pv_beamline(0.0, 0.0, 0.0, 0.0)
    h = ctypes.c_void_p()
    assert lib.pv_init(ctypes.byref(cfg), ctypes.byref(beam), 0, ctypes.byref(h)) == pv.PV_ERR_ARG
    assert not h.value


def test_strerror(lib):
    import paper_2412_14966_gb300 as pv
    assert pv.load().pv_strerror(0) == b"ok"
    assert pv.load().pv_strerror(pv.PV_ERR_BUSY) == b"busy"


def test_product_path_does_not_import_the_oracle():
    """The package and its build never import or read oracle/ (it is test
    infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2412_14966_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "oracle/" not in src, f
                assert "pv_oracle" not in src, f


def test_default_build_has_no_bounds_checks(lib):
    """pv_check_report answers PV_ERR_ARG with zeros in the default build (no
    device call is made)."""
    import paper_2412_14966_gb300 as pv
    assert pv.check_report() == (False, 0, 0)


def test_checked_build_compiles_with_the_same_exports():
    """The checked test build (PV_CHECKED=1) compiles for sm_103a and exports
    every function the header declares."""
    from paper_2412_14966_gb300 import build
    path = build.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    names = set(re.findall(r"\bpv_\w+", out))
    declared = set(re.findall(r"\b(pv_\w+)\s*\(", open(HEADER).read()))
    assert declared <= names, declared - names
