"""The C-ABI library builds, loads and exports every entry point declared in
include/lrp.h, and the Python binding's structures match the C layouts
(no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1703_05638_gb300 as lrp
from paper_1703_05638_gb300 import build as lrp_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lrp.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lrp_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    lrp_build.build()
    return lrp.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "lrp_hessian_apply" in names and "lrp_lowrank_posterior" in names
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps exactly the declared set
    assert sorted(lrp.EXPORTS) == names


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lrp.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(lrp_problem_desc), sizeof(lrp_apply_stats), sizeof(lrp_lanczos_stats),'
                   'sizeof(lrp_query), sizeof(lrp_query_result), offsetof(lrp_problem_desc, mg_nu_coarse),'
                   'offsetof(lrp_query, xi), sizeof(lrp_tuning), offsetof(lrp_tuning, last_team_ctas));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(lrp.lrp_problem_desc), ctypes.sizeof(lrp.lrp_apply_stats),
            ctypes.sizeof(lrp.lrp_lanczos_stats), ctypes.sizeof(lrp.lrp_query),
            ctypes.sizeof(lrp.lrp_query_result), lrp.lrp_problem_desc.mg_nu_coarse.offset,
            lrp.lrp_query.xi.offset, ctypes.sizeof(lrp.lrp_tuning), lrp.lrp_tuning.last_team_ctas.offset]
    assert got == want


def test_version_and_error_strings(lib):
    assert lrp.lrp_version().startswith("lrpost-gb300")
    assert isinstance(lrp.lrp_last_error(), str)


def test_sources_have_no_host_fallback():
    """The product path is the CUDA library only: the binding never imports
    the oracle, and every compute entry point goes through liblrp.so."""
    src = open(os.path.join(ROOT, "paper_1703_05638_gb300", "__init__.py")).read()
    assert "oracle" not in src.replace("the oracle", "")
    assert "import scipy" not in src


def test_server_struct_layouts_match_c(tmp_path):
    names = ["lrp_server_config", "lrp_request_stats", "lrp_server_stats", "lrp_tuning", "lrp_als_stats",
             "lrp_arnoldi_stats", "lrp_problem_desc"]
    src = tmp_path / "sz2.c"
    body = "".join(f'printf("%zu\\n", sizeof({n}));' for n in names)
    src.write_text('#include <stdio.h>\n#include "lrp.h"\nint main(void){' + body + 'return 0;}\n')
    exe = tmp_path / "sz2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [ctypes.sizeof(getattr(lrp, n)) for n in names]
