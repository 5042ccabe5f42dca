"""The C-ABI library builds, loads and exports every declared symbol (CPU only)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_10032_gb300 import build
    build.build()
    from paper_2503_10032_gb300 import ddelm
    return ddelm


def _declared():
    src = open(os.path.join(ROOT, "include", "ddelm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(ddelm_\w+)\s*\(", src, re.M)))


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert set(declared) == set(lib.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared:
        assert re.search(rf"\bT {name}\b", out), name


def test_query_matches_oracle_layout(lib):
    from oracle.layout import Layout
    from paper_2503_10032_gb300 import inputs
    for p in [inputs.small_problem(3, 2, M=9, n_int=20, edge_pts=3), inputs.config("poisson_2x2_m100"),
              inputs.small_problem(4, 1, M=5, n_int=10, edge_pts=2)]:
        sz = lib.ddelm_query(lib.ProblemArgs(p, lib.make_options()))
        lay = Layout(p.nx, p.ny, p.box, p.edge_pts)
        assert (sz.n_pi, sz.n_delta, sz.n_bnd) == (lay.n_pi, lay.n_delta, lay.n_bnd)
        assert sz.sum_M == p.M.sum() and sz.sum_int == p.n_int.sum()
        assert sz.workspace_bytes > 0


def test_invalid_arguments_are_rejected(lib):
    from paper_2503_10032_gb300 import inputs
    p = inputs.small_problem(2, 2, M=6, n_int=10, edge_pts=2)
    pa = lib.ProblemArgs(p, lib.make_options(theta=1.5))
    with pytest.raises(lib.DDELMError):
        lib.ddelm_query(pa)
    p.M[0] = 0
    with pytest.raises(lib.DDELMError):
        lib.ddelm_query(lib.ProblemArgs(p, lib.make_options()))
    assert lib.ddelm_status_string(lib.DDELM_ERR_TIMEOUT).startswith("a device")
