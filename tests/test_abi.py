"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/stiv.h (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "stiv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(stiv_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("stiv_upsample", "stiv_detect", "stiv_stiv", "stiv_stiv_grad", "stiv_grad_to_coef", "stiv_step"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1812_04719_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_1812_04719_gb300 import stiv
    assert sorted(stiv.EXPORTS) == declared_functions()


def test_status_strings_without_gpu():
    from paper_1812_04719_gb300 import stiv
    assert stiv.status_string(0) == "ok"
    assert "capacity" in stiv.status_string(2)


def test_static_sort_limit_matches_header():
    from paper_1812_04719_gb300 import stiv
    src = open(os.path.join(ROOT, "include", "stiv.h")).read()
    m = re.search(r"#define\s+STIV_SORT_STATIC_MAX\s+\(1 << (\d+)\)", src)
    assert m and stiv.SORT_STATIC_MAX == 1 << int(m.group(1))
