"""The CUDA library loads without a GPU and exports every entry point that
include/lbmib.h declares (no compute calls)."""
import os
import re

from paper_2607_07432_b300 import lbmib

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbmib.h")


def declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:lbm_status|void|const char\*|long long)\s+(\w+)\s*\(", src, re.M)))


def test_header_matches_binding_list():
    assert declared() == sorted(lbmib.EXPORTS)


def test_library_exports_all_symbols():
    lib = lbmib.load()
    for name in declared():
        assert hasattr(lib, name), name


def test_config_default_without_gpu():
    import ctypes as ct
    lib = lbmib.load()
    cfg = lbmib.Config()
    assert lib.lbm_config_default(ct.byref(cfg)) == 0
    assert cfg.struct_size == ct.sizeof(lbmib.Config)
    assert abs(cfg.sigma_hrr - 0.98) < 1e-15 and abs(cfg.d_n - 1.5) < 1e-15
    assert lib.lbm_config_default(None) == 1
