"""The C-ABI library builds for sm_103a and exports every entry point include/ozk.h declares
(no GPU needed: only loading and symbol lookup)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ozk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libozk():
    from paper_2603_29975_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ozaki_zgemm", "ozaki_zgemm_vbatched", "ozk_zgemm_dmma", "kkr_tau00", "kkr_tau00_batched",
                 "kkr_build_m", "ozk_split_debug", "ozk_group_sums_debug", "ozk_create", "ozk_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libozk):
    for name in _declared():
        assert hasattr(libozk, name), name


def test_binding_lists_every_export():
    from paper_2603_29975_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_argument_errors_need_no_gpu(libozk):
    libozk.ozk_zgemm_workspace_size.restype = ctypes.c_size_t
    assert libozk.ozk_zgemm_workspace_size(512, 512, 512, 7, 1) > 7 * 512 * 1024 * 2
    assert libozk.ozk_zgemm_workspace_size(512, 512, 512, 17, 1) == 0       # S out of range
    assert libozk.ozaki_zgemm(None, b"N", b"N", 1, 1, 1, None, None, 1, None, 1, None, None, 1, 7, 0) == 1


def test_binding_constants_match_the_header():
    from paper_2603_29975_gb300 import binding
    src = open(os.path.join(ROOT, "include", "ozk.h")).read()
    defs = dict(re.findall(r"^#define (OZK_[A-Z0-9_]+) (\d+)\b", src, flags=re.M))
    checked = [k for k in defs if hasattr(binding, k)]
    assert {"OZK_NB_MAX", "OZK_SEL_NPARAMS", "OZK_SEL_FEATURES", "OZK_PAIRS_FULL"} <= set(checked)
    for k in checked:
        assert getattr(binding, k) == int(defs[k]), k
