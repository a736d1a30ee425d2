"""The C ABI without a GPU: libdme.so builds for sm_103a, loads, exports every
function include/dme.h declares, and the Python descriptor matches the C
struct layout.  No compute call is made."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1805_08990_gb300 as dme
from paper_1805_08990_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    return build.build()


def test_library_exports_every_declared_function(libpath):
    names = binding.header_functions()
    assert {"dme_plan", "dme_expm", "dme_step", "dme_solve", "dme_submit", "dme_poll"} <= set(names)
    L = ctypes.CDLL(libpath)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    r = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    if r.returncode == 0:
        exported = {ln.split()[-1] for ln in r.stdout.splitlines() if ln.strip()}
        assert set(names) <= exported


def test_binding_signatures_cover_header():
    assert set(binding.header_functions()) == set(binding._SIGS)


def test_desc_layout_matches_c_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "layout.c"
    fields = [f for f, _ in binding.dme_plan_desc._fields_]
    body = "\n".join(f'printf("{f} %zu\\n", offsetof(dme_plan_desc, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dme.h"\nint main(void){\n'
                   + body + '\nprintf("size %zu\\n", sizeof(dme_plan_desc));\nreturn 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = dict(zip(out[0::2], map(int, out[1::2])))
    for f in fields:
        assert got[f] == getattr(binding.dme_plan_desc, f).offset, f
    assert got["size"] == ctypes.sizeof(binding.dme_plan_desc)


def test_header_is_plain_c(tmp_path):
    """include/dme.h compiles as C99 and as C++ with no CUDA or torch types."""
    txt = open(os.path.join(ROOT, "include", "dme.h")).read()
    assert "torch" not in txt and "cuda_runtime" not in txt
    src = tmp_path / "h.c"
    src.write_text('#include "dme.h"\nint main(void){ return (int)sizeof(dme_plan_desc) > 0 ? 0 : 1; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(tmp_path / "h")], check=True)


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(binding, "LIB_PATH", "/nonexistent/libdme.so")
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(dme.LibraryNotBuilt):
        binding.lib()


def test_make_desc_fields():
    d = dme.make_desc(7, m=2, p=3, eq=dme.DME_DRE, comp="lie", flows=("F1", "F3", "F2"), h=0.25,
                      q_is_factor=True)
    assert (d.n, d.m, d.p, d.eq, d.comp, d.nflows) == (7, 2, 3, dme.DME_DRE, dme.DME_LIE, 3)
    assert list(d.flows)[:3] == [dme.DME_F1, dme.DME_F3, dme.DME_F2]
    assert d.h == 0.25 and d.q_is_factor == 1


def test_enum_values_follow_the_boundary_table(tmp_path):
    """dme_prec keeps the boundary's numbering: FP64 = 0, SPLIT_TF32 = 1 (reserved,
    rejected), SPLIT_BF16 = 2; the binding's constants match the C header."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    names = ["DME_FP64", "DME_SPLIT_TF32", "DME_SPLIT_BF16", "DME_DLE", "DME_DRE", "DME_GDLE", "DME_GDRE",
             "DME_F1", "DME_F2", "DME_F12", "DME_F3", "DME_F4", "DME_LIE", "DME_STRANG", "DME_OK", "DME_EINVAL",
             "DME_ENOTREADY"]
    src = tmp_path / "enums.c"
    body = "\n".join(f'printf("{n} %d\\n", (int){n});' for n in names)
    src.write_text('#include <stdio.h>\n#include "dme.h"\nint main(void){\n' + body + '\nreturn 0;}\n')
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = dict(zip(out[0::2], map(int, out[1::2])))
    assert (got["DME_FP64"], got["DME_SPLIT_TF32"], got["DME_SPLIT_BF16"]) == (0, 1, 2)
    for n in names:
        assert got[n] == getattr(binding, n), n
