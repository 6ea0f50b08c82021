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


def test_flags_and_order_limit_match_header():
    """The binding's status flags and order limit are the header's and the
    library's."""
    from paper_1812_04719_gb300 import stiv
    src = open(os.path.join(ROOT, "include", "stiv.h")).read()
    for name in ("PAIRS_OVERFLOW", "CONTACTS_OVERFLOW", "BOX_TOO_SMALL", "NONFINITE", "WORK_OVERFLOW", "TIMEOUT",
                 "BAD_ORDER"):
        m = re.search(r"STIV_F_%s\s*=\s*(\d+)" % name, src)
        assert m and getattr(stiv, "F_" + name) == int(m.group(1)), name
    cuh = open(os.path.join(ROOT, "paper_1812_04719_gb300", "csrc", "stiv_internal.cuh")).read()
    m = re.search(r"#define\s+STIV_MAX_P\s+(\d+)", cuh)
    assert m and stiv.MAX_ORDER == int(m.group(1))


def test_bad_order_rejected_on_host():
    """Orders outside [1, 32] never reach the device from the binding."""
    import numpy as np
    from paper_1812_04719_gb300 import scenegen as G
    from paper_1812_04719_gb300 import stiv
    for bad in (0, 33):
        sc = G.scene_small((2, 1, 1), p=4, seed=3)
        sc.p = sc.p.copy()
        sc.p[1] = bad
        try:
            stiv.DeviceScene.from_scene(sc, device="cpu")
        except ValueError as e:
            assert "[1, 32]" in str(e)
        else:
            raise AssertionError(bad)
    assert np.asarray(sc.p).dtype.kind == "i"
