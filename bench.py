#!/usr/bin/env python
"""DDELM-NN solves/sec on GB300.

One step = one pass of the whole path on one problem: the setup (feature
assembly, factorisation of every local least-squares problem, local and
coarse operators) followed by one solve (right-hand side of Eq. nn-mixed, CG
to the relative residual tolerance, reconstruction by Eq. coarse_sol_2).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Under torchrun every rank solves its own independent replica of the problem
(no data-path collective; weak scaling); rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DDELM solves/sec to rel. interface residual 1e-8 (mixed vs FP64, same GB300)"
DEFAULT_WORKLOAD = "poisson_8x8_m400"
TOL = 1e-8
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07
EPS_REL = 1e-8
THETA = 0.999

# DRAM traffic of the slice-GEMM class (dram__bytes_read.sum + dram__bytes_write.sum),
# taken once with ncu (one pass) over the 26 launches of one step of the default
# workload, and valid only for the kernel and plan sources it was taken on: the
# bench reports it (per launch, like "achieved") only when their hash matches.
TC_TRAFFIC = {
    "workload": "poisson_8x8_m400",
    "dram_bytes_per_step": 15824769536 + 2952566528,
    "launches_per_step": 26,
    "sources_sha256": "f6b4696adf81ef5ccc5333a6f58a9b7cd09c228739554440fbea621e862accf3",
    "source": ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
               "--clock-control none -k regex:ozaki_gemm_all -s 26 -c 26 python bench.py --steps 1 --warmup 3 "
               "--no-cpu-baseline --no-fp64-compare --solve-steps 0 (second setup; per launch = step / 26)"),
}
TC_SOURCES = ("paper_2503_10032_gb300/csrc/ozaki_tc.cu", "paper_2503_10032_gb300/csrc/ozaki_plan.cpp",
              "paper_2503_10032_gb300/csrc/plan.cpp")


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for f in TC_SOURCES:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()
FP64_PEAK_GFLOPS = 1250.0   # GB300 nominal FP64: 152 SMs x 4 FLOP/clk x 2.07 GHz
SCHEMES = {"auto": 0, "fp64cqr3": 1, "fp32": 2, "cqr2series": 3, "cqr2series-dw": 4}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def method_setup_flops(sub_sizes):
    """The method's algorithmic setup work per step (what DDELM-NN has to compute,
    not what this implementation executes).  Per subdomain with m rows, M neurons,
    nG interface and nDl Delta points: the Gram of the m - nG interior and
    boundary rows shared by K_c and K-bar ((m - nG) M^2, symmetric), the Grams of
    the two interface blocks (2 nG M^2), the three local operators Lambda, Psi,
    Phi (triangular solves and products: 2 nG M^2 + 3 nG^2 M + 2 nDl M^2 +
    2 nDl^2 M) and two Cholesky factorisations (2 M^3 / 3).  Returns (GEMM flops,
    Cholesky flops)."""
    gemm = chol = 0.0
    for d in sub_sizes:
        m, M, nG, nDl = (float(d[k]) for k in ("m", "M", "nG", "nDl"))
        gemm += (m - nG) * M * M + 2 * nG * M * M + 2 * nG * M * M + 3 * nG * nG * M + 2 * nDl * M * M \
            + 2 * nDl * nDl * M
        chol += 2.0 * M ** 3 / 3.0
    return gemm, chol


def workload_config(name, prob, sizes=None):
    cfg = {"workload": name, "subdomains": f"{prob.nx}x{prob.ny}",
           "neurons_per_subdomain": int(prob.M[0]) if len(set(prob.M.tolist())) == 1 else "uneven",
           "interior_points_per_subdomain": int(prob.n_int[0]) if len(set(prob.n_int.tolist())) == 1 else "uneven",
           "points_per_edge": int(prob.edge_pts[0]) if len(set(prob.edge_pts.tolist())) == 1 else "uneven",
           "n_rhs": int(prob.n_rhs), "theta": THETA, "eps_rel": EPS_REL, "tol": TOL,
           "operator": "poisson" if prob.op == 0 else "diffusion"}
    if sizes is not None:
        cfg["n_pi"] = int(sizes.n_pi)
        cfg["n_delta"] = int(sizes.n_delta)
    return cfg


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_complete_solve(prob):
    """Times one complete FP64 oracle solve of the workload: every local ridge
    pseudo-inverse by Householder QR, the coarse problem (S_Pi assembled and
    factored), plain CG on Eq. (nn-mixed) from mu = 0 to the relative residual
    TOL, and the reconstruction of Eq. (coarse_sol_2) with u at the evaluation
    points.  Returns (seconds, CG iterations)."""
    from oracle import ddelm as odd
    t0 = time.perf_counter()
    r = odd.solve(prob, odd.Options(eps_rel=EPS_REL, theta=THETA, tol=TOL), method="cg")
    return time.perf_counter() - t0, int(r["iters"])


def oracle_threads():
    """Threads the oracle's BLAS runs with (its parallelism is BLAS-level)."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count() or 1


def max_over_ranks(x, dist, device):
    """The maximum of x over the ranks of the job (x itself on one process):
    the whole-job time is the slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """The oracle on the host cores: every timed step is one complete oracle solve
    of the workload (see oracle_complete_solve); the warm-up steps solve the 2x2,
    M = 100 workload completely (imports, BLAS threads and caches warmed at a
    fraction of the cost)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2503_10032_gb300 import inputs
    prob = inputs.config(args.workload)
    small = inputs.config("poisson_2x2_m100")
    for _ in range(args.warmup):
        oracle_complete_solve(small)
    per, its = [], []
    for _ in range(args.steps):
        dt, it = oracle_complete_solve(prob)
        per.append(dt)
        its.append(it)
    sec = float(np.mean(per))
    value = 1.0 / sec
    cores = oracle_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, prob),
            "cg_iterations": int(np.median(its)),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step one complete FP64 oracle solve of the whole workload "
                                       f"({prob.n_sub} local ridge pseudo-inverses by Householder QR, coarse "
                                       f"problem, CG to relative residual {TOL}, reconstruction); warm-up "
                                       f"steps solve the 2x2, M=100 workload"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    global THETA
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scheme", default="auto", choices=list(SCHEMES))
    ap.add_argument("--passes", type=int, default=0, help="FP32 scheme: shifted passes (0: automatic)")
    ap.add_argument("--solve-steps", type=int, default=5, help="timed solves with the reused handle")
    ap.add_argument("--tc-tiles", type=int, default=0, choices=[0, 1, 2, 3],
                    help="MIXED tensor-core tile shapes: 0 all-levels by rule + autotuner, "
                         "1 level-group shapes only, 2 all-levels only, 3 128x64 level groups only")
    ap.add_argument("--theta", type=float, default=THETA,
                    help="NN weight of Eq. (nn-mixed); 0 gives the coarse-space method without the NN term")
    args = ap.parse_args()
    THETA = args.theta
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2503_10032_gb300 import build as _b
    _b.build()
    from paper_2503_10032_gb300 import ddelm as D
    from paper_2503_10032_gb300 import inputs

    prob = inputs.config(args.workload)
    prec = D.DDELM_PREC_FP64 if args.precision == "fp64" else D.DDELM_PREC_MIXED
    opt_kw = dict(theta=THETA, eps_rel=EPS_REL, tol=TOL, max_iters=20000, precision=prec,
                  setup_scheme=SCHEMES[args.scheme], setup_passes=args.passes, tc_tiles=args.tc_tiles)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        solver = D.Solver(prob, device=dev, stream=stream, **opt_kw)
        f = torch.tensor(prob.f_int, dtype=torch.float64, device=dev)
        g = torch.tensor(prob.g_bnd, dtype=torch.float64, device=dev)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    sizes = solver.sizes
    sub_sizes = []
    for i_ in range(sizes.n_sub):
        m_, M_, nG_, nDl_ = D.ddelm_inspect(solver.h, i_, 7, 4)
        sub_sizes.append({"m": m_, "M": M_, "nG": nG_, "nDl": nDl_})
    flops = D.ddelm_inspect(solver.h, 0, 8, 7)
    plan = D.ddelm_inspect(solver.h, 0, 9, 4)
    scheme_desc = {1: "fp64-cholesky-cqr3", 3: "fp64-cholesky x2 + series", 4: "double-fp32-cholesky x2 + series"}.get(
        int(plan[0]), f"fp32-cholesky x{int(plan[1])} shifted + 1 polished")

    def step():
        solver.refactor()
        return solver.solve(f, g)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize(dev)
    plan6 = D.ddelm_inspect(solver.h, 0, 9, 6)
    graphs = {"setup": bool(plan6[4]), "solve": bool(plan6[5])}

    def timed_steps(n):
        """n steps between CUDA events on the library's stream, L2 flushed before
        each (outside the events); returns (per-step ms, solve infos)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        res = []
        for k in range(n):
            with torch.cuda.stream(stream):
                flush.zero_()                         # L2 flush, outside the timed events
                ev[k][0].record(stream)
            o = step()
            ev[k][1].record(stream)
            res.append((o[3].iterations, o[3].rel_residual, o[4], o))
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in ev], res

    # timed region: the production configuration (setup and solve replayed from
    # their captured CUDA graphs, no per-launch events)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    step_ms, res = timed_steps(args.steps)
    barrier()
    clk = clocks.stop()
    infos = [r[:3] for r in res]
    out = res[-1][3]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, dist, dev)
    value = world * args.steps / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # profiled pass: the same number of steps again with CUDA events around every
    # launch (graphs are not replayed while profiling), for the per-kernel-class
    # times, launch counts and the roofline of the dominant class
    solver.profile(enable=True, reset=True)
    prof_step_ms, _ = timed_steps(args.steps)
    prof_ms, prof_n = solver.profile(enable=False, reset=True)

    # secondary metric: repeated solves with the reused handle (right-hand side,
    # CG and reconstruction only), L2 flushed between solves
    solve_only = None
    if args.solve_steps > 0:
        evs = []
        for k in range(args.solve_steps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.zero_()
                a0.record(stream)
            o_s = solver.solve(f, g)
            a1.record(stream)
            evs.append((a0, a1))
        torch.cuda.synchronize(dev)
        ts = float(sum(a.elapsed_time(b_) for a, b_ in evs))
        solve_only = {"value": world * args.solve_steps / (ts / 1e3), "unit": "solves/s",
                      "ms_per_solve": ts / args.solve_steps, "steps": args.solve_steps,
                      "cg_iterations": int(o_s[3].iterations), "rel_residual": float(o_s[3].rel_residual)}

    # the same steps on the FP64 path (the metric compares mixed with FP64 on the same GPU)
    fp64_cmp = None
    if args.precision == "mixed" and not args.no_fp64_compare:
        with torch.cuda.stream(stream):
            s64 = D.Solver(prob, device=dev, stream=stream,
                           **dict(opt_kw, precision=D.DDELM_PREC_FP64, setup_scheme=0, setup_passes=0))
        for _ in range(1):
            s64.refactor()
            o64 = s64.solve(f, g)
        torch.cuda.synchronize(dev)
        ev64 = []
        for k in range(args.steps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.zero_()
                a0.record(stream)
            s64.refactor()
            o64 = s64.solve(f, g)
            a1.record(stream)
            ev64.append((a0, a1))
        torch.cuda.synchronize(dev)
        t64 = float(sum(a.elapsed_time(b_) for a, b_ in ev64))
        u_mixed = out[2].double().cpu().numpy()
        u64 = o64[2].double().cpu().numpy()
        fp64_cmp = {"value": args.steps / (t64 / 1e3), "ms_per_step": t64 / args.steps,
                    "cg_iterations": int(o64[3].iterations), "rel_residual": float(o64[3].rel_residual),
                    "mixed_vs_fp64_rel_l2_u": float(np.linalg.norm(u_mixed - u64) / max(np.linalg.norm(u64), 1e-300))}
        s64.close()
        del s64

    # end to end through the C ABI with host buffers: setup from host arrays,
    # H2D of the data from pinned memory, solve, D2H of c, mu and u
    f_h = torch.tensor(prob.f_int, dtype=torch.float64).pin_memory()
    g_h = torch.tensor(prob.g_bnd, dtype=torch.float64).pin_memory()
    R = prob.n_rhs
    c_h = torch.empty((sizes.sum_M, R), dtype=torch.float64).pin_memory()
    mu_h = torch.empty((sizes.n_pi + sizes.n_delta, R), dtype=torch.float64).pin_memory()
    u_h = torch.empty((max(sizes.sum_eval, 1), R), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    e2e_ms = []
    ws_ptr, ws_bytes = solver.ws_ptr, int(sizes.workspace_bytes)
    pa = D.ProblemArgs(prob, D.make_options(**opt_kw))
    tune = D.ddelm_inspect(solver.h, 0, 11, 4 + 5 * 128)   # the tile-shape autotuner's outcome
    solver.close()
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, h, _ = D.ddelm_setup(pa, ws_ptr, ws_bytes, stream.cuda_stream)
        if rc != D.DDELM_OK:
            raise D.DDELMError(rc, "ddelm_setup (e2e)")
        with torch.cuda.stream(stream):
            f_d = f_h.to(dev, non_blocking=True)
            g_d = g_h.to(dev, non_blocking=True)
            c_d = torch.empty((sizes.sum_M, R), dtype=torch.float64, device=dev)
            mu_d = torch.empty((sizes.n_pi + sizes.n_delta, R), dtype=torch.float64, device=dev)
            u_d = torch.empty((max(sizes.sum_eval, 1), R), dtype=torch.float64, device=dev)
        rc, info = D.ddelm_solve(h, f_d.data_ptr(), g_d.data_ptr(), c_d.data_ptr(), mu_d.data_ptr(),
                                 u_d.data_ptr(), stream.cuda_stream)
        with torch.cuda.stream(stream):
            c_h.copy_(c_d, non_blocking=True)
            mu_h.copy_(mu_d, non_blocking=True)
            u_h.copy_(u_d, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        D.ddelm_destroy(h)
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = float(sum(e2e_ms))
    e2e_total = max_over_ranks(e2e_total, dist, dev)
    e2e_value = world * e2e_steps / (e2e_total / 1e3)
    h2d = int(sizes.upload_bytes) + f_h.numel() * 8 + g_h.numel() * 8
    d2h = c_h.numel() * 8 + mu_h.numel() * 8 + u_h.numel() * 8

    # roofline of the dominant kernel class: the method's algorithmic work per
    # step over the class's time per step in the profiled pass
    names = D.PROF_CLASS_NAMES
    n_cls = len(names)
    launches_total = int(prof_n.sum())
    peaks = measured_peaks()
    alg_gemm, alg_chol = method_setup_flops(sub_sizes)
    # the method's GEMM work is split between the tensor-core and FP64 engines in
    # the proportion of the implementation's own (FP64-equivalent) setup products
    tc_share = (flops[0] - flops[4]) / flops[0] if (prec == D.DDELM_PREC_MIXED and flops[0] > 0) else 0.0
    bf16_peak = 1000.0 * float(peaks.get("bf16_tflops_sustained", 1700.0))
    bf16_src = "bf16_tflops_sustained of MEASURED_PEAKS.json (kernel timed inside a long step)"
    alg_work = {"tc_gemm": alg_gemm * tc_share, "gemm_f64": alg_gemm * (1.0 - tc_share) + flops[2],
                "chol_inv": alg_chol}
    # the roofline is the method's algorithmic work over the time of the class
    # that does it: the largest of the classes that carry that work
    k_dom = max((i for i, n in enumerate(names) if n in alg_work), key=lambda i: prof_ms[i])
    dom = names[k_dom]
    per_launch_ms = prof_ms[k_dom] / max(prof_n[k_dom], 1)
    work_per_launch = alg_work.get(dom, float("nan")) * args.steps / max(prof_n[k_dom], 1)
    bound, unit, peak, peak_src = "alu", "GFLOP/s", FP64_PEAK_GFLOPS, \
        "nominal FP64 of the recipe table (no FP64 entry in the measured peaks)"
    if dom == "tc_gemm":
        bound, peak, peak_src = "tensor", bf16_peak, bf16_src
    elif dom == "chol_inv" and flops[5] > 0.5 * flops[1]:
        peak, peak_src = FP32_PEAK_GFLOPS, ("nominal FP32 CUDA-core rate (152 SMs x 128 lanes x 2 x 2.07 GHz); "
                                            "the Cholesky passes run in FP32")
    achieved = work_per_launch / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else float("nan")
    traffic = None
    if (dom == "tc_gemm" and args.workload == TC_TRAFFIC["workload"] and prec == D.DDELM_PREC_MIXED
            and args.scheme == "auto" and args.tc_tiles == 0
            and kernel_sources_sha256() == TC_TRAFFIC["sources_sha256"]):
        traffic = TC_TRAFFIC["dram_bytes_per_step"] / TC_TRAFFIC["launches_per_step"]
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak if math.isfinite(achieved) else None,
                "traffic": traffic, "traffic_source": TC_TRAFFIC["source"] if traffic is not None else None,
                "peak_source": peak_src,
                "work": ("the method's algorithmic setup flops per step (per subdomain: shared Gram, two "
                         "interface updates, three local operators; two Cholesky factorisations for chol_inv)"
                         f" = {alg_gemm:.4g} GEMM + {alg_chol:.4g} Cholesky flops, times the class's share; "
                         "per launch = per step x steps / launches"),
                "time_share": {n: float(prof_ms[i] / max(prof_ms[:n_cls].sum(), 1e-12)) for i, n in enumerate(names)},
                "launches": {n: int(prof_n[i]) for i, n in enumerate(names)},
                "profiled_ms_per_step": float(np.mean(prof_step_ms))}
    if dom == "tc_gemm":
        # what the tensor cores execute: the BF16 slice-pair products of the exact
        # FP64 emulation (far more than the method's flops)
        emu = flops[3] * args.steps / (prof_ms[k_dom] * 1e-3) / 1e9
        roofline["emulated"] = {"achieved": emu, "peak": bf16_peak, "unit": "GFLOP/s", "frac": emu / bf16_peak,
                                "work": "BF16 slice-pair flops executed per step", "flops_per_step": flops[3]}
        roofline["vs_fp64_nominal"] = {"peak": FP64_PEAK_GFLOPS, "frac": achieved / FP64_PEAK_GFLOPS,
                                       "note": "the same algorithmic rate against the nominal FP64 rate"}

    # every kernel class against its own roof (algorithmic work over live time)
    n_it = float(np.median([i for i, _, _ in infos]))
    cg_bytes = 8.0 * n_it * sum(3.0 * s_["nG"] ** 2 + 2.0 * s_["nDl"] ** 2 for s_ in sub_sizes) \
        + 8.0 * n_it * 8.0 * sizes.n_pi ** 2
    feat_bytes = 8.0 * sum((2 * s_["m"] + s_["nG"] + s_["nDl"]) * s_["M"] for s_ in sub_sizes)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    roofs = {"features": (feat_bytes, "GB/s", hbm, "hbm (matrix bytes written; the tanh arithmetic is FP64)"),
             "gemm_f64": (alg_work["gemm_f64"], "GFLOP/s", FP64_PEAK_GFLOPS, "alu (FP64 nominal)"),
             "chol_inv": (alg_chol, "GFLOP/s", FP32_PEAK_GFLOPS if flops[5] > 0.5 * flops[1] else FP64_PEAK_GFLOPS,
                          "alu (FP32 nominal)" if flops[5] > 0.5 * flops[1] else "alu (FP64 nominal)"),
             "cg_persistent": (cg_bytes, "GB/s", hbm, "hbm (local operators read per iteration)"),
             "slicing": (flops[6], "GB/s", hbm, "hbm"),
             "tc_gemm": (alg_work["tc_gemm"], "GFLOP/s", bf16_peak,
                         "tensor (BF16 sustained, measured); the method's flops")}
    kernels = {}
    for i, n in enumerate(names):
        if n not in roofs or prof_ms[i] <= 0:
            continue
        w, u_, pk, kind = roofs[n]
        ach = w * args.steps / (prof_ms[i] * 1e-3) / 1e9
        kernels[n] = {"achieved": ach, "unit": u_, "peak": pk, "frac": ach / pk, "bound": kind,
                      "ms_per_step": prof_ms[i] / args.steps}

    iters = [i for i, _, _ in infos]
    resid = max(r for _, r, _ in infos)
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16x9+f64",
            "data": "synthetic",
            "config": dict(workload_config(args.workload, prob, sizes), precision=args.precision,
                           factorisation=scheme_desc, setup_waves=int(plan[2]),
                           tc_tiles=["all-levels 128x48 by rule, autotuned against level groups",
                                     "level groups 128x64 / 128x128", "all-levels 128x48",
                                     "level groups 128x64"][args.tc_tiles],
                           parallelism=f"replicas{world}", l2="flushed between steps (512 MB write)"),
            "cg_iterations": int(np.median(iters)), "rel_residual_max": resid,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "gpu_launches": launches_total, "roofline": roofline, "kernels": kernels, "clocks": clk}
    if solve_only is not None:
        line["solve_only"] = solve_only
    if fp64_cmp is not None:
        line["fp64"] = fp64_cmp
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # one complete oracle solve of the workload when its dense local
        # pseudo-inverses fit comfortably in host memory (the 8x8, M = 400
        # workload: about 30 s on 16 cores); larger workloads are not sampled
        oracle_bytes = 8.0 * sum(4.0 * d["m"] * d["M"] for d in sub_sizes)
        if oracle_bytes < 8e9:
            dt, it = oracle_complete_solve(prob)
            line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "solves/s", "cores": oracle_threads(),
                                    "kind": "oracle", "cg_iterations": it,
                                    "sample": f"one complete FP64 oracle solve of the whole workload ({dt:.1f} s): "
                                              f"{prob.n_sub} local ridge pseudo-inverses by Householder QR, coarse "
                                              f"problem, CG to relative residual {TOL}, reconstruction"}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": oracle_threads(), "kind": "oracle",
                                    "sample": f"not run: the oracle's dense local pseudo-inverses need "
                                              f"{oracle_bytes / 1e9:.0f} GB"}
    line["gpu_launches_source"] = ("kernel launches of the library counted in the profiled pass (the same "
                                   f"{args.steps} steps as the timed region, whose captured graphs replay them)")
    line["graphs"] = graphs
    line["autotune"] = {"phases_timed": int(tune[0]), "switched": int(tune[1]),
                        "ms_rule_widths": float(tune[2]), "ms_chosen_widths": float(tune[3]),
                        "phases": [[int(tune[4 + 5 * k]), int(tune[5 + 5 * k]), round(float(tune[6 + 5 * k]), 4),
                                    int(tune[7 + 5 * k]), round(float(tune[8 + 5 * k]), 4)]
                                   for k in range(min(int(tune[0]), 128)) if tune[5 + 5 * k] > 0],
                        "note": "tensor-core tile width per GEMM phase, timed on the handle's first setup; "
                                "phases: [index, rule width, ms, alternative width, ms]"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
