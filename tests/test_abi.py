"""The C-ABI library loads and exports every entry point include/mdx.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

from paper_2405_01834_gb300 import build, mdx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "mdx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mdx_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = declared()
    for need in ("mdx_create", "mdx_destroy", "mdx_last_error", "mdx_sync", "mdx_eri4", "mdx_eri3", "mdx_schwarz"):
        assert need in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    for name in declared():
        assert hasattr(lib, name), name


def test_planner_covers_every_class():
    """Every 4-center class up to l = 6 and every 3-center class plans and passes the
    planner's shared-memory bounds checks (host only)."""
    for la in range(7):
        for lb in range(7):
            for lc in range(7):
                for ld in range(lc, 7):
                    st = mdx.plan_info(la, lb, lc, ld)
                    assert st.smem_bytes_per_team <= 227 * 1024
                    assert st.team_threads * st.teams_per_cta <= 1024
        for lc in range(7):
            for ld in range(7):
                mdx.plan_info(la, 0, lc, ld, 1, 1, True)


def test_planner_contracted_and_rejects():
    st = mdx.plan_info(0, 0, 0, 0, 36, 36)
    assert st.exec_fma > 0
    mdx.plan_info(2, 1, 1, 0, 18, 6)
    with pytest.raises(mdx.MdxError):
        mdx.plan_info(7, 0, 0, 0)
    with pytest.raises(mdx.MdxError):
        mdx.plan_info(1, 1, 1, 1, 0, 1)
    with pytest.raises(mdx.MdxError):
        mdx.plan_info(1, 1, 1, 1, 1, 1, True)   # one-centre bra needs lb = 0
