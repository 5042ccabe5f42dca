"""Comparison helpers shared by the parity tests.

Every comparison of a GPU result with the oracle checks two numbers: the
relative L2 distance |a - b| / |b| and the element-wise distance
max |a - b| / max |b| (an error confined to a few entries, e.g. one
subdomain of many, shows in the second even when the norm hides it).  The
norm-wise tolerances come from the spread of two backward-stable FP64
factorisations of the same ridge problems; the element-wise bound is a fixed
multiple of it (ENTRYWISE_FACTOR).  When
the environment variable PARITY_LOG names a file, every comparison appends a
JSON line with both numbers, so a run reports the attained parity.
"""
import json
import os

import numpy as np


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0


ENTRYWISE_FACTOR = 4.0


def close(a, b, tol, what="", tol_max=None):
    """True when the relative L2 distance is below tol and the element-wise one
    below tol_max (default ENTRYWISE_FACTOR x tol: measured entry-wise, the
    spread of two backward-stable FP64 factorisations of the same ridge problems
    (Householder QR vs SVD pseudo-inverses) is up to 2.7x its norm-wise value,
    since the largest entries of a smooth field exceed its root mean square);
    logs both."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    r2, rm = rel_l2(a, b), rel_max(a, b)
    path = os.environ.get("PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"what": what, "rel_l2": r2, "rel_max": rm, "tol": tol,
                                "tol_max": ENTRYWISE_FACTOR * tol if tol_max is None else tol_max}) + "\n")
    tm = ENTRYWISE_FACTOR * tol if tol_max is None else tol_max
    ok = r2 < tol and rm < tm
    if not ok:
        print(f"parity {what}: rel_l2 {r2:.3e} rel_max {rm:.3e} tol {tol:.1e} / {tm:.1e}")
    return ok


def load_golden(path_no_ext):
    """A stored oracle result: <name>.txt or <name>.txt.gz."""
    for ext in (".txt", ".txt.gz"):
        if os.path.exists(path_no_ext + ext):
            return np.loadtxt(path_no_ext + ext, ndmin=2)
    raise FileNotFoundError(path_no_ext)
