"""The C-ABI library builds, loads without a GPU, and exports every symbol of include/*.h."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(occ_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_hot_path():
    names = _declared_functions()
    for n in ("occ_trace_ao", "occ_trace_shadow", "occ_reuse_ao", "occ_reuse_shadow",
              "occ_bvh_build", "occ_create", "occ_sync"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2607_23122_gb300 import _native
    lib = _native.load()
    names = _declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for each symbol, and nothing else
    assert sorted(_native.SIGNATURES) == names


def test_version_and_no_gpu_errors_are_clean():
    from paper_2607_23122_gb300 import _native
    lib = _native.load()
    assert b"sm_103a" in lib.occ_version()
    h = ctypes.c_void_p()
    st = lib.occ_create(0, ctypes.byref(h))
    import torch
    if not torch.cuda.is_available():
        assert st != 0 and not h.value     # no device: a clean error, no crash
    else:
        assert st == 0
        lib.occ_destroy(h)


def test_struct_layouts_match_the_header():
    """Sizes of the ctypes mirrors equal the C structs (LP64)."""
    from paper_2607_23122_gb300 import _native as N
    assert ctypes.sizeof(N.occ_gbuffer) == 40
    assert ctypes.sizeof(N.occ_rect_light) == 36
    assert ctypes.sizeof(N.occ_pattern) == 40
    assert ctypes.sizeof(N.occ_bvh_stats) == 48
    # W H format (pad) data effect radius light(36) (pad) seed sample (pad)
    assert ctypes.sizeof(N.occ_occluders) == 88
    assert ctypes.sizeof(N.occ_sched_config) == 24
    assert ctypes.sizeof(N.occ_sched_stats) == 72
    assert ctypes.sizeof(N.occ_server_config) == 48
    assert ctypes.sizeof(N.occ_tuning) == 36
    # W H effect radius light(36) (pad) seed sample (pad) pattern(40) K estimator packed
    # camera(40) eps 4 pointers deadline
    assert ctypes.sizeof(N.occ_request) == 208
    assert ctypes.sizeof(N.occ_result) == 40
    assert ctypes.sizeof(N.occ_server_stats) == 112
