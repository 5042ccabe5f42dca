"""Writes the FP64 oracle's results on the full-size workloads for the parity
tests of the CUDA path.  Calls the oracle only; the inputs (problems, seeded
interface vectors) come from the seeded generator module.

Every workload uses theta = 0.999 and eps_rel = 1e-8 (the benchmark's launch
configuration), the Sec. 3 structured method with S_theta of Eq. (nn-mixed)
assembled by applying the operator to unit vectors and solved by Cholesky
(an exact solve of Eq. (nn-mixed), no iteration error), then Eq. (coarse_sol_2).

  poisson_8x8_m400          mu on Delta, u at the evaluation points, and the
                            operator check (below)
  poisson_16x16_uneven      the same
  diffusion_4x4_m1000_r16   the same (the 32x32 workload's per-subdomain shape)
  poisson_8x8_grf           the same (g = 0, f a GRF with alpha = 32, Sec. 4.3)
  varcoef_8x8_grf           the same (-div(rho grad u) = 1, rho = tanh(GRF) + 1.1, Sec. 4.4)
  biharmonic_16x16          the same (Lap^2 u = f, u = Lap u = 0 on the boundary, Sec. 4.5:
                            256 subdomains, M = 256, a 20 x 20 grid, l = 64; the
                            system in u and v = Lap u / s^2)
  poisson_8x8_fourier       U = du/da (u at the evaluation points for each of the
                            16 Fourier modes as forcing, g = 0: u is linear in a),
                            and dL/ds for two losses by a fourth-order central
                            difference of the oracle's solution at s + j h,
                            j = -2, -1, 1, 2, at eps_rel 1e-4 and 1e-6

Operator check: S_theta mu_k for two seeded N(0, 1) interface vectors mu_k
(inputs.interface_vectors(n_delta, n_rhs, 2, seed 7001)), and b_theta.

    python tests/golden/make_fullsize_golden.py [workload ...]
"""
import dataclasses
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ddelm as odd  # noqa: E402
from paper_2503_10032_gb300 import inputs  # noqa: E402

OPTS = dict(theta=0.999, eps_rel=1e-8)
MU_SEED = 7001
SCALE_STEP = 1e-3          # relative step of the scale difference
SOLUTION_SETS = ("poisson_8x8_m400", "poisson_16x16_uneven", "diffusion_4x4_m1000_r16", "poisson_8x8_grf",
                 "varcoef_8x8_grf", "biharmonic_16x16")


def _save(name, what, arr, head):
    path = os.path.join(HERE, f"{name}_{what}.txt" + (".gz" if np.asarray(arr).size > 20000 else ""))
    np.savetxt(path, np.asarray(arr).reshape(np.asarray(arr).shape[0], -1), fmt="%.17e", header=head)
    print("wrote", path, flush=True)


def solution_set(name):
    p = inputs.config(name)
    t0 = time.time()
    o = odd.DDELMOracle(p, odd.Options(**OPTS))
    head = (f"FP64 oracle, {name}: theta 0.999, eps_rel 1e-8, S_theta assembled and solved by Cholesky")
    mu, S, b = o.solve_direct()
    cs, _ = o.reconstruct(mu)
    u = o.u_eval(cs)
    _save(name, "mu_delta", mu, head + "; mu on the Delta points [n_delta x n_rhs]")
    _save(name, "u_eval", u, head + "; u at the evaluation points [n_eval x n_rhs]")
    vs = inputs.interface_vectors(o.n_dl, p.n_rhs, 2, MU_SEED)
    outs = [o.S_theta_apply(v) for v in vs]
    _save(name, "S_apply", np.hstack(outs),
          head + f"; S_theta mu_k for mu_k = inputs.interface_vectors(n_delta, n_rhs, 2, {MU_SEED}), "
                 "columns [k * n_rhs + r]")
    _save(name, "b_theta", b, head + "; b_theta [n_delta x n_rhs]")
    print(name, f"{time.time() - t0:.0f} s", flush=True)


def fourier_set(with_u=True):
    name = "poisson_8x8_fourier"
    p = inputs.config(name)
    t0 = time.time()
    if with_u:
        # U: the 16 modes as 16 right-hand sides (g = 0)
        q = inputs.config(name)
        q.f_int = inputs.fourier_basis(q.x_int)
        q.g_bnd = np.zeros((q.g_bnd.shape[0], 16))
        o = odd.DDELMOracle(q, odd.Options(**OPTS))
        mu, S, b = o.solve_direct()
        cs, _ = o.reconstruct(mu)
        U = o.u_eval(cs)
        head = f"FP64 oracle, {name}: theta 0.999, eps_rel 1e-8, direct solve"
        _save(name, "dU_da", U, head + "; u at the evaluation points for forcing = mode (p, q), g = 0 "
                                       "[n_eval x 16], column 4 (p-1) + (q-1)")
    # dL/ds: the loss's dependence on s is far below the rounding level of the
    # solution at eps_rel = 1e-8 (|u| changes by ~1e-12 for a 1e-3 step), so the
    # scale derivative is taken at eps_rel = 1e-4 and 1e-6, where a fourth-order
    # central difference of the oracle's solution is accurate; two losses: the
    # workload's L1 = mean (u - sin(pi x) sin(pi y))^2 and L2 = sum w_k u_k with
    # seeded N(0, 1) weights w (inputs.interface_vectors(n_eval, 1, 1, 7002)).
    target = np.sin(np.pi * p.x_eval[:, 0]) * np.sin(np.pi * p.x_eval[:, 1])
    wts = inputs.interface_vectors(len(target), 1, 1, 7002)[0][:, 0]
    h = SCALE_STEP * p.scale
    rows = []
    for eps in (1e-4, 1e-6):
        vals = {}
        for j in (-2, -1, 1, 2):
            r = dataclasses.replace(p, scale=p.scale + j * h)
            oo = odd.DDELMOracle(r, odd.Options(theta=0.999, eps_rel=eps))
            m, _, _ = oo.solve_direct()
            c2, _ = oo.reconstruct(m)
            ue = oo.u_eval(c2)[:, 0]
            vals[j] = (float(np.mean((ue - target) ** 2)), float(wts @ ue))
            print("eps", eps, "scale step", j, vals[j], flush=True)
        for k in range(2):
            d4 = (-vals[2][k] + 8 * vals[1][k] - 8 * vals[-1][k] + vals[-2][k]) / (12 * h)
            d2 = (vals[1][k] - vals[-1][k]) / (2 * h)
            rows.append([eps, k + 1, d4, d2, h])
    head = (f"FP64 oracle, {name}: theta 0.999, direct solves; rows [eps_rel, loss (1: mean (u - sin(pi x) "
            f"sin(pi y))^2, 2: sum w_k u_k with w = inputs.interface_vectors(n_eval, 1, 1, 7002)), dL/ds by the "
            f"fourth-order central difference at s + j h (j = -2, -1, 1, 2), dL/ds by the second-order one "
            f"(j = -1, 1), h = {SCALE_STEP} s]; f = sum a_pq mode_pq with a = inputs.fourier_coefficients(), g = 0")
    _save(name, "dL_ds", np.array(rows), head)
    print(name, f"{time.time() - t0:.0f} s", flush=True)


def main():
    which = sys.argv[1:] or list(SOLUTION_SETS) + ["poisson_8x8_fourier"]
    for name in which:
        if name == "poisson_8x8_fourier":
            fourier_set()
        elif name == "poisson_8x8_fourier_scale":
            fourier_set(with_u=False)
        else:
            solution_set(name)


if __name__ == "__main__":
    main()
