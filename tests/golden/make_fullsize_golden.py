"""Writes the FP64 oracle's solution of the 8x8-subdomain, M=400 Poisson workload
(u = sin 2 pi x cos 3 pi y, theta = 0.999, eps_rel = 1e-8) for the full-size
parity test: mu on the Delta points and u at the evaluation points.  Calls the
oracle only; the inputs come from the seeded generator module.

    python tests/golden/make_fullsize_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ddelm as odd  # noqa: E402
from paper_2503_10032_gb300 import inputs  # noqa: E402

NAME = "poisson_8x8_m400"


def main():
    p = inputs.config(NAME)
    r = odd.solve(p, odd.Options(theta=0.999, eps_rel=1e-8), method="direct")
    head = f"FP64 oracle, {NAME}: theta 0.999, eps_rel 1e-8, S_theta assembled and solved directly"

    np.savetxt(os.path.join(HERE, f"{NAME}_mu_delta.txt"), np.asarray(r["mu_delta"]), fmt="%.17e",
               header=head + "; mu on the Delta points [n_delta x n_rhs]")
    np.savetxt(os.path.join(HERE, f"{NAME}_u_eval.txt"), np.asarray(r["u_eval"]), fmt="%.17e",
               header=head + "; u at the evaluation points [n_eval x n_rhs]")


if __name__ == "__main__":
    main()
