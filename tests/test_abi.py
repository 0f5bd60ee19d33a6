"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point of include/alifmm.h."""
import ctypes
import os
import re

from paper_2302_10988_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "alifmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(alf_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_header_symbols():
    lib = build.build()
    L = ctypes.CDLL(lib)
    names = _header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(binding.EXPORTS) == names


def test_default_options_without_gpu():
    o = binding.alf_default_options()
    assert o.precision == binding.ALF_FP32 and o.init_radius == 2 and o.plane_step == 4
    assert o.stop_radius == 1.6 and o.band_cells > 0


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    try:
        binding.alf_create(0)
    except binding.AlfError as e:
        assert e.code == 4  # ALF_ERR_CUDA: no device
    else:
        raise AssertionError("alf_create succeeded without a GPU")
