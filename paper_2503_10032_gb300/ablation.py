"""The paper's ablation on the GPU (Sec. 4.2): CG iterations and the solution's
error for the coarse-space variants of Table 1 ({K, K_c} x {A, A_m}, without
the Neumann-Neumann term (theta = 0, Eq. (coarse_sol_1)) and with it
(theta = 1, Eq. (nn))) and for the mixing weight theta of Table 2 (K_c, A_m),
on the paper's problem u = sin(pi x) sin(pi y) at the paper's scale
(inputs.paper_scale; the 2x2 and 4x4 grids are capped at 1024 neurons per
subdomain).  CG runs to the paper's relative residual 1e-9.

    python -m paper_2503_10032_gb300.ablation [--grids 2,4,8,16] [--precision fp64|mixed]
    python -m paper_2503_10032_gb300.ablation --table6 [--grids 2,4,8,16]
    python -m paper_2503_10032_gb300.ablation --levels

--levels: what the BF16-slice level counts of the MIXED setup buy.  On the
8x8 / M = 400 workload each class of tensor-core products (Grams after the
first pass, Q and ridge-block updates, products of triangular factors, local
operators and their inputs, the first Gram) loses 1, 2 or 3 slice levels in
turn; each run reports whether the setup succeeds, the relative L2 distances
of u, mu and the local operator Lambda^0 from the FP64 path (the parity
tolerances on this workload: u 1e-7, local operators 1e-6 sampled and S_theta
1e-7; their measured FP64 spread ~1e-8) and the GPU time of one setup + solve.

Prints one JSON line per solve and the two tables in markdown.  --table6: the
biharmonic problem of Sec. 4.5 (Lap^2 u = f, u = Lap u = 0 on the boundary,
u = sin(pi x) sin(pi y), l = 64) solved by vanilla DDELM (no coarse space),
DDELM-CS (theta = 0) and DDELM-NN (theta = 0.999, K_c and A_m), with the GPU
time of one setup + solve.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

VARIANTS = [("K, A", False, False), ("K_c, A", True, False), ("K, A_m", False, True), ("K_c, A_m", True, True)]
THETAS = [0.0, 0.5, 0.9, 0.99, 0.999, 0.9999, 1.0]


def run_one(D, prob, torch, timed=False, **kw):
    s = D.Solver(prob, **kw)
    f = torch.tensor(prob.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(prob.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    out = {}
    if timed:
        # one more setup + solve on the same handle, timed with events on the current stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.refactor()
        c, mu, u, info, rc = s.solve(f, g)
        e1.record()
        torch.cuda.synchronize()
        out["setup_solve_ms"] = float(e0.elapsed_time(e1))
    u = u.cpu().numpy()[:, 0]
    ex = prob.u_eval_exact[:, 0]
    err = float(np.linalg.norm(u - ex) / np.linalg.norm(ex))
    s.close()
    return dict(iterations=int(info.iterations), rel_residual=float(info.rel_residual), status=int(rc),
                rel_l2_error=err, **out)


LEVEL_CLASSES = [(16, "first Gram"), (1, "Grams after the first pass"), (2, "Q and ridge-block updates"),
                 (4, "products of triangular factors"), (8, "local operators and their inputs")]


def levels(D, torch, args):
    from . import inputs
    prob = inputs.config("poisson_8x8_m400")
    common = dict(eps_rel=1e-8, tol=1e-8, theta=0.999)
    f = torch.tensor(prob.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(prob.g_bnd, dtype=torch.float64, device="cuda")

    def run(**kw):
        s = None
        try:
            s = D.Solver(prob, **common, **kw)
            s.solve(f, g)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.refactor()
            c, mu, u, info, rc = s.solve(f, g)
            e1.record()
            torch.cuda.synchronize()
            lam = s.inspect(0, 3)   # Lambda^0, a local operator
            return ((u.cpu().numpy(), mu.cpu().numpy(), lam), float(e0.elapsed_time(e1)),
                    "ok" if rc == D.DDELM_OK else "not converged")
        except D.DDELMError as e:
            return None, None, str(e).split(":")[1].strip()
        finally:
            if s is not None:
                s.close()
    ref, _, _ = run(precision=D.DDELM_PREC_FP64)

    def dist(out):
        if out is None:
            return [float("nan")] * 3
        return [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(out, ref)]
    base, base_ms, _ = run(precision=D.DDELM_PREC_MIXED)
    rows = [("none", 0, dist(base), base_ms, "ok")]
    for mask, name in LEVEL_CLASSES:
        for trim in (1, 2, 3):
            out, ms, st = run(precision=D.DDELM_PREC_MIXED, trim_levels=trim, trim_mask=mask)
            d = dist(out)
            rows.append((name, trim, d, ms, st))
            print(json.dumps(dict(levels=name, trim=trim, u=d[0], mu=d[1], Lambda0=d[2], setup_solve_ms=ms,
                                  status=st)), flush=True)
    print("\n| class | levels removed | u | mu | Lambda^0 | setup + solve (ms) | status |")
    print("|---|---|---|---|---|---|---|")
    for name, trim, d, ms, st in rows:
        print(f"| {name} | {trim} | {d[0]:.1e} | {d[1]:.1e} | {d[2]:.1e} | "
              f"{ms if ms is not None else float('nan'):.1f} | {st} |")


def table6(D, torch, grids, prec, args):
    """Sec. 4.5: DDELM, DDELM-CS and DDELM-NN on the biharmonic problem."""
    from . import inputs
    rows = {}
    for n in grids:
        prob = inputs.paper_scale(n, op=inputs.OP_BIHARMONIC)
        nG = 2 * (4 * (320 // n) + 4)
        p = prec if nG <= 256 else D.DDELM_PREC_FP64   # MIXED holds at most 256 interface rows per subdomain
        for name, kw in (("DDELM", dict(theta=0.0, use_coarse=False)), ("DDELM-CS", dict(theta=0.0)),
                         ("DDELM-NN", dict(theta=0.999))):
            r = run_one(D, prob, torch, timed=True, eps_rel=args.eps_rel, tol=1e-9, max_iters=args.max_iters,
                        precision=p, **kw)
            r["precision"] = "fp64" if p == D.DDELM_PREC_FP64 else "mixed"
            rows[(name, n)] = r
            print(json.dumps(dict(table=6, grid=f"{n}x{n}", M=int(prob.M[0]), method=name, **r)), flush=True)
    print("\nTable 6 (biharmonic, u = sin(pi x) sin(pi y))\n")
    print("| method | grid | M | rel. L2 error | iterations | setup + solve (ms) | precision |")
    print("|---|---|---|---|---|---|---|")
    for (name, n), r in sorted(rows.items(), key=lambda kv: (kv[0][0], kv[0][1])):
        print(f"| {name} | {n}x{n} | {min(2 ** 16 // (n * n), 1024)} | {r['rel_l2_error']:.2e} | {r['iterations']} | "
              f"{r['setup_solve_ms']:.1f} | {r['precision']} |")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--grids", default="2,4,8,16")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--eps-rel", type=float, default=1e-8)
    ap.add_argument("--max-iters", type=int, default=60000)
    ap.add_argument("--table6", action="store_true")
    ap.add_argument("--levels", action="store_true")
    args = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    from . import ddelm as D
    from . import inputs
    prec = D.DDELM_PREC_FP64 if args.precision == "fp64" else D.DDELM_PREC_MIXED
    grids = [int(x) for x in args.grids.split(",")]
    if args.table6:
        table6(D, torch, grids, prec, args)
        return 0
    if args.levels:
        levels(D, torch, args)
        return 0
    t1, t2 = {}, {}
    for n in grids:
        prob = inputs.paper_scale(n)
        common = dict(eps_rel=args.eps_rel, tol=1e-9, max_iters=args.max_iters, precision=prec)
        for name, cov, am in VARIANTS:
            for theta in (0.0, 1.0):
                r = run_one(D, prob, torch, theta=theta, use_change_of_vars=cov, use_Am=am, **common)
                t1[(name, theta, n)] = r
                print(json.dumps(dict(table=1, grid=f"{n}x{n}", M=int(prob.M[0]), variant=name, theta=theta, **r)),
                      flush=True)
        for theta in THETAS:
            r = run_one(D, prob, torch, theta=theta, **common)
            t2[(theta, n)] = r
            print(json.dumps(dict(table=2, grid=f"{n}x{n}", M=int(prob.M[0]), theta=theta, **r)), flush=True)
    head = "| " + " | ".join(f"{n}x{n} err / iter" for n in grids) + " |"
    print("\nTable 1 (theta 0: coarse space only; theta 1: with the Neumann-Neumann term)\n")
    print("| variant | theta " + head)
    print("|---|---|" + "---|" * len(grids))
    for name, _, _ in VARIANTS:
        for theta in (0.0, 1.0):
            cells = [f"{t1[(name, theta, n)]['rel_l2_error']:.2e} / {t1[(name, theta, n)]['iterations']}" for n in grids]
            print(f"| {name} | {theta:g} | " + " | ".join(cells) + " |")
    print("\nTable 2 (K_c, A_m)\n")
    print("| theta " + head)
    print("|---|" + "---|" * len(grids))
    for theta in THETAS:
        cells = [f"{t2[(theta, n)]['rel_l2_error']:.2e} / {t2[(theta, n)]['iterations']}" for n in grids]
        print(f"| {theta:g} | " + " | ".join(cells) + " |")
    return 0


if __name__ == "__main__":
    sys.exit(main())
