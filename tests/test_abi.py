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


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's size and field offsets (a field added
    to one side only, or in another order, would corrupt every call that passes the struct)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = [binding.alf_material, binding.alf_options, binding.alf_stats, binding.alf_geometry]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "alifmm.h"', "int main(void) {"]
    for S in structs:
        lines.append(f'  printf("{S.__name__} size %zu\\n", sizeof({S.__name__}));')
        for f in S._fields_:
            lines.append(f'  printf("{S.__name__} {f[0]} %zu\\n", offsetof({S.__name__}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for S in structs:
        assert got[(S.__name__, "size")] == ctypes.sizeof(S), S.__name__
        for f in S._fields_:
            assert got[(S.__name__, f[0])] == getattr(S, f[0]).offset, (S.__name__, f[0])


def test_new_sweep_options_default_to_the_plans_choice():
    o = binding.alf_default_options()
    assert o.cta_threads == 0 and o.cta_cluster == 0 and o.sweep == 0 and o.velocity_table == 0
