"""Host-side checks of the C ABI (no GPU needed): the library builds and
exports every function declared in include/refusion.h, the binding declares
the same set, and host-side argument handling works without a device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1905_02082_gb300 import build as B
    return B.build()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "refusion.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(rf_[a-z_]+)\s*\(", text))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("rf_create_volume", "rf_track_frame", "rf_integrate_frame", "rf_extract_mesh", "rf_compute_mask",
              "rf_process_frame", "rf_volume_export", "rf_volume_import", "rf_destroy_volume", "rf_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rf_[a-z_]+)\b", out))
    missing = _declared_functions() - exported
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in _declared_functions():
        getattr(lib, n)


def test_binding_covers_every_declared_symbol():
    import paper_1905_02082_gb300.refusion as R
    assert {s[0] for s in R.SIGNATURES} == _declared_functions()


def test_default_params_are_table_1(lib_path):
    import json
    import paper_1905_02082_gb300.refusion as R
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "tab1_parameters.json")))
    p = R.rf_default_params()
    for k in ("voxel_size", "trunc", "w_c", "theta", "gamma"):
        assert getattr(p, k) == g[k]


def test_struct_sizes_match_header(lib_path, tmp_path):
    """ctypes layouts equal the C layouts (compiled with the host compiler)."""
    import paper_1905_02082_gb300.refusion as R
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "refusion.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(rf_params), sizeof(rf_frame),'
                   ' sizeof(rf_track_info), sizeof(rf_stats), offsetof(rf_params, max_candidates));'
                   'printf("%zu\\n", sizeof(rf_profile));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    assert got == [ctypes.sizeof(R.rf_params), ctypes.sizeof(R.rf_frame), ctypes.sizeof(R.rf_track_info),
                   ctypes.sizeof(R.rf_stats), R.rf_params.max_candidates.offset, ctypes.sizeof(R.rf_profile)]


def test_argument_errors_are_reported_on_the_host(lib_path):
    import paper_1905_02082_gb300.refusion as R
    lib = R.load()
    p = R.rf_default_params()
    h = ctypes.c_void_p()
    # invalid parameters are rejected before any CUDA call
    bad = R.rf_default_params()
    bad.voxel_size = 0.0123456789
    assert lib.rf_create_volume(ctypes.byref(bad), 1 << 10, 100, 64, 64, ctypes.byref(h)) == 1
    assert b"micrometre" in lib.rf_last_error(None)
    assert lib.rf_create_volume(ctypes.byref(p), 1000, 100, 64, 64, ctypes.byref(h)) == 1  # not a power of two
    assert lib.rf_create_volume(None, 1 << 10, 100, 64, 64, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.rf_destroy_volume(None) == 0
    assert lib.rf_track_frame(None, None, None, None, None, None, None) == 1
    assert lib.rf_status_string(3) == b"hash table full"


def test_volume_footprint_without_a_device(lib_path):
    """rf_volume_footprint needs no GPU and charges exactly the per-block and
    per-bucket storage: a block is 512 voxels x (8 B value/colour word + 1 B
    weight) + its coordinates (16 B) + its neighbour table (32 B); a bucket is
    4 slots x 8 B."""
    import paper_1905_02082_gb300.refusion as R
    p = R.rf_default_params()
    base = R.rf_volume_footprint(p, 1 << 12, 1000, 640, 480)
    assert R.rf_volume_footprint(p, 1 << 12, 1001, 640, 480) - base == 512 * 9 + 16 + 32
    assert R.rf_volume_footprint(p, 1 << 13, 1000, 640, 480) - base == (1 << 12) * 4 * 8
    # per-pixel scratch grows with the frame bound
    assert R.rf_volume_footprint(p, 1 << 12, 1000, 1280, 720) > base
    with pytest.raises(R.RFError):
        R.rf_volume_footprint(p, 1000, 1000, 640, 480)  # buckets not a power of two
    with pytest.raises(R.RFError):
        R.rf_volume_footprint(p, 1 << 12, 0, 640, 480)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the built library the binding raises; it has no fallback."""
    import paper_1905_02082_gb300.refusion as R
    monkeypatch.setattr(R, "_lib", None)
    with pytest.raises(ImportError):
        R.load(str(tmp_path / "librefusion.so"))


def test_batch_rejects_closed_volumes_and_mismatched_lists():
    """Checked in the binding before anything reaches the library."""
    import types
    import paper_1905_02082_gb300.refusion as R
    b = R.Batch.__new__(R.Batch)
    b.volumes = [types.SimpleNamespace(h=1), types.SimpleNamespace(h=None)]
    b.h = 1
    with pytest.raises(R.RFError):
        b.process([None, None], [None, None], [None, None])
    b.volumes[1].h = 2
    with pytest.raises(R.RFError):
        b.process([None], [None, None], [None, None])
    b.h = None  # nothing to release


def test_binding_checks_image_arguments():
    import numpy as np
    import torch
    import paper_1905_02082_gb300.refusion as R
    d = torch.zeros(4, 6, dtype=torch.int16)
    with pytest.raises(ValueError):  # pageable host memory
        R.make_frame(d, torch.zeros(4, 6, 3, dtype=torch.uint8), 1.0, 1.0, 2.0, 2.0)
    with pytest.raises(ValueError):  # wrong colour shape
        R.make_frame(d, torch.zeros(4, 6, dtype=torch.uint8), 1.0, 1.0, 2.0, 2.0)
    T = np.eye(4)
    with pytest.raises(ValueError):  # float depth
        R.rf_process_frame_host(None, np.zeros((4, 6)), np.zeros((4, 6, 3), np.uint8), [1, 1, 2, 2], T, T.copy())
    with pytest.raises(ValueError):  # float32 pose
        R.rf_process_frame_host(None, np.zeros((4, 6), np.uint16), np.zeros((4, 6, 3), np.uint8), [1, 1, 2, 2],
                                T.astype(np.float32), T.copy())
