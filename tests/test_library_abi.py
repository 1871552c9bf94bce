"""The CUDA library loads without a GPU and exports every entry point that
include/*.h declares (no compute calls)."""
import glob
import os
import re

from paper_2607_07432_b300 import lbmib, nop

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared(name="*.h"):
    out = set()
    for h in glob.glob(os.path.join(INC, name)):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        out |= set(re.findall(r"^\s*(?:lbm_status|void|const char\*|long long)\s+(\w+)\s*\(", src, re.M))
    return sorted(out)


def test_header_matches_binding_list():
    assert declared("lbmib.h") == sorted(lbmib.EXPORTS)
    assert declared("nop.h") == sorted(nop.NOP_EXPORTS)


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
    # defaults: central a^C stencil (reading Q6), no artificial bulk viscosity (Q29)
    assert cfg.use_ac == lbmib.AC_CENTRAL and cfg.bulk_ratio == 0.0
    assert lib.lbm_config_default(None) == 1


def test_nop_config_default_without_gpu():
    import ctypes as ct
    cfg = nop.NopConfig()
    L = nop._lib()
    assert L.nop_config_default(ct.byref(cfg)) == 0
    assert cfg.struct_size == ct.sizeof(nop.NopConfig)
    assert (cfg.height, cfg.width, cfg.in_channels, cfg.out_channels) == (256, 512, 3, 4)
    assert list(cfg.channels) == [32, 64, 96, 128]
    assert L.nop_create(None, None) == 1
