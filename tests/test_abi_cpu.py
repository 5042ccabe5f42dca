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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_workload_plans(lib, prec):
    """The host plan of every workload passes its own bounds and shape checks
    (every kernel access, tensor-map box and tile range) in both precisions."""
    from paper_2503_10032_gb300 import inputs
    pr = lib.DDELM_PREC_FP64 if prec == "fp64" else lib.DDELM_PREC_MIXED
    for name in inputs.CONFIGS:
        sz = lib.ddelm_query(lib.ProblemArgs(inputs.config(name), lib.make_options(precision=pr)))
        assert sz.workspace_bytes > 0, name


def test_rejection_names_the_check(lib):
    from paper_2503_10032_gb300 import inputs
    p = inputs.small_problem(2, 2, M=6, n_int=10, edge_pts=2)
    with pytest.raises(lib.DDELMError, match="theta must be in"):
        lib.ddelm_query(lib.ProblemArgs(p, lib.make_options(theta=1.5)))
