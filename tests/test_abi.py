"""C-ABI library checks that need no GPU: it builds, loads, exports every
entry point that include/epic.h declares, and rejects bad descriptions on
the host before touching a device."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1603_02126_gb300 import _binding as B
    return B.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "epic.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(epic_\w+|epical_\w+)\s*\(", txt)))


def test_header_declares_expected_calls():
    names = _declared()
    for must in ("epic_plan_create", "epic_image", "epical_update", "epical_configure",
                 "epic_plan_destroy", "epic_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1603_02126_gb300 import _binding as B
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTS) == _declared()


def _desc(B, **over):
    ant = np.array([[0.0, 0.0], [3.0, 1.0], [-2.0, 4.0]])
    freq = np.array([50e6])
    keep = dict(ant=ant, freq=freq)
    d = B.PlanDesc()
    d.n_ant = 3
    d.ant_xy_m = ant.ctypes.data_as(B.c_dp)
    d.n_chan = 1
    d.freq_hz = freq.ctypes.data_as(B.c_dp)
    d.grid_n = 32
    d.cell_wavelengths = 0.5
    d.kernel = 0
    d.kernel_support = 3
    d.kernel_param = 0.5
    d.input = 0
    d.precision = 0
    for k, v in over.items():
        if k == "ant":
            a = np.ascontiguousarray(v, np.float64)
            keep["ant2"] = a
            d.ant_xy_m = a.ctypes.data_as(B.c_dp)
            d.n_ant = a.shape[0]
        elif k == "kernel_param_ant":
            a = np.ascontiguousarray(v, np.float64)
            keep["kpa"] = a
            d.kernel_param_ant = a.ctypes.data_as(B.c_dp)
        else:
            setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("over,code", [
    (dict(grid_n=48), 1),
    (dict(grid_n=8), 1),
    (dict(kernel_support=4), 1),
    (dict(kernel_param=-1.0), 1),
    (dict(cell_wavelengths=0.0), 1),
    (dict(input=7), 1),
    (dict(precision=5), 1),
    (dict(precision=1, path=1), 7),
    (dict(grid_n=1024), 7),
    (dict(ant=[[60.0, 0.0], [0.0, 0.0]]), 2),
    (dict(path=5), 1),                      # unknown path
    (dict(kernel_param_ant=[0.5, -1.0, 0.5]), 1),   # per-antenna parameters must be > 0
    (dict(path=4, grid_n=32), 7),           # warp-specialised form: N = 64 or 128 only
    (dict(path=4, precision=2), 7),         # ... and FP32 only
    (dict(path=3, grid_n=128), 7),          # cluster form: N = 256 or 512 only
    (dict(path=3, grid_n=256, precision=1), 7),
])
def test_create_rejects_on_host(lib, over, code):
    from paper_1603_02126_gb300 import _binding as B
    d, keep = _desc(B, **over)
    h = ct.c_void_p()
    st = lib.epic_plan_create(ct.byref(h), ct.byref(d))
    assert st == code, lib.epic_last_error()
    assert h.value is None
    assert lib.epic_last_error().decode()


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.epic_image(None, None, 1, None, 0) == 1
    assert lib.epical_update(None, None, None) == 1
    assert lib.epical_average_channels(None, 0, 1) == 1
    assert lib.epic_plan_destroy(None) == 0


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the descriptor, info and tune-result structs
    have the sizes and field offsets a C compiler gives include/epic.h."""
    import shutil
    import subprocess
    from paper_1603_02126_gb300 import _binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"epic_plan_desc": B.PlanDesc, "epic_plan_info": B.PlanInfo,
               "epic_tune_result": B.TuneResult}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "epic.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ct.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
