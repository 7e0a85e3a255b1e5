"""Host-side checks of the C-ABI library (no GPU needed).

libmrirecon.so must build for sm_103a, load, and export every function that
include/mrirecon.h declares; argument validation that happens before any
device work must reject bad input with MRI_ERR_INVALID.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrirecon.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_14080_gb300 import build
    path = build.build()
    import paper_2006_14080_gb300 as mr
    return mr.load(path)


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"MRI_API\s+[\w\s\*]+?\b(mri_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mri_plan_create", "mri_plan_destroy", "mri_nudft_forward", "mri_nudft_adjoint",
                     "mri_normal_op", "mri_tv_forward", "mri_tv_adjoint", "mri_admm_reconstruct"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(mri_\w+)", out))
    assert set(declared_functions()) <= exported
    # nothing else leaks out with the mri_ prefix
    assert exported <= set(declared_functions())


def test_host_side_validation(lib):
    assert lib.mri_version() >= 100
    h = ctypes.c_void_p()
    assert lib.mri_plan_create(None, 4, 4, 4, 1, None, 0, None) == -1
    assert lib.mri_plan_create(ctypes.byref(h), -3, 4, 4, 1, ctypes.c_void_p(16), 0, None) == -1
    assert b"positive" in lib.mri_last_error()
    assert lib.mri_plan_create(ctypes.byref(h), 4, 4, 4, 1, None, 0, None) == -1
    assert lib.mri_tv_forward(0, 4, None, None, None) == -1
    assert lib.mri_soft_threshold(-1, 0.5, None, None, None) == -1
    assert lib.mri_plan_destroy(None) == 0
    assert lib.mri_plan_device_bytes(None) == 0


def test_tuning_table_round_trip(lib, tmp_path):
    import paper_2006_14080_gb300 as mr
    src = tmp_path / "tuned.json"
    src.write_text('{"format": "mrirecon-tuning", "version": 1, "entries": [\n'
                   ' {"precision": 2, "nx": 128, "ny": 128, "nk": 16384, "nc": 12, "sms": 152,'
                   ' "fwd_coils_per_tile": 2, "fwd_stages": 3, "adj_stages": 3},\n'
                   ' {"precision": 1, "nx": 256, "ny": 256, "nk": 65536, "nc": 32, "sms": 152,'
                   ' "fwd_coils_per_tile": 1, "fwd_stages": 2, "adj_stages": 2}\n]}\n')
    mr.tuning_clear()
    assert mr.tuning_count() == 0
    mr.tuning_load(str(src))
    assert mr.tuning_count() == 2
    out = tmp_path / "saved.json"
    mr.tuning_save(str(out))
    mr.tuning_clear()
    mr.tuning_load(str(out))
    assert mr.tuning_count() == 2
    again = tmp_path / "again.json"
    mr.tuning_save(str(again))
    assert again.read_text() == out.read_text()
    # malformed files are rejected without touching the table
    bad = [('{"format": "other"}', "not a tuning file"),
           ('{"format": "mrirecon-tuning", "entries": [{"precision": 2, "nx": 8}]}', "without integer"),
           ('{"format": "mrirecon-tuning", "entries": [{"precision": 2, "nx": 8, "ny": 8, "nk": 8, "nc": 1,'
            ' "sms": 152, "fwd_coils_per_tile": 5, "fwd_stages": 3, "adj_stages": 3}]}', "coils per tile"),
           ('{"format": "mrirecon-tuning", "entries": [{"precision": 2, "nx": 8, "ny": 8, "nk": 8, "nc": 1,'
            ' "sms": 152, "fwd_coils_per_tile": 1, "fwd_stages": 5, "adj_stages": 3}]}', "stage count")]
    for text, why in bad:
        f = tmp_path / "bad.json"
        f.write_text(text)
        with pytest.raises(mr.MriError) as ei:
            mr.tuning_load(str(f))
        assert ei.value.code == mr.MRI_ERR_INVALID and why in str(ei.value)
        assert mr.tuning_count() == 2
    with pytest.raises(mr.MriError):
        mr.tuning_load(str(tmp_path / "missing.json"))
    mr.tuning_clear()
