"""Seeded synthetic DDELM problems (inputs only; no part of the method's arithmetic).

A problem is the data of the 2-D PDE and of its decomposition that the paper's
method takes as given (Sec. 2.1, Sec. 2.2.1, Sec. 4.1): the rectangle and its
nx x ny grid of subdomains, the hidden-layer parameters of every local network
(w = s * w_hat, b = s * b_hat), the interior collocation points, the number of
equispaced points on every grid edge, the forcing f at the interior points and
the Dirichlet data g at the boundary points, plus evaluation points.

Geometry conventions that every consumer implements on its own:

* subdomain (ix, iy) has index iy*nx + ix and covers
  [x0 + ix*hx, x0 + (ix+1)*hx] x [y0 + iy*hy, y0 + (iy+1)*hy];
* grid vertices (vx, vy), 0 <= vx <= nx, 0 <= vy <= ny;
* horizontal edge (ix, vy) joins vertices (ix, vy) and (ix+1, vy), id vy*nx + ix;
  vertical edge (vx, iy) joins (vx, iy) and (vx, iy+1), id nx*(ny+1) + vx*ny + iy;
* edge E with e points carries them at start + k/(e+1) * (end - start),
  k = 1..e, start being the vertex with the smaller coordinate;
* the global list of Dirichlet points is: for every edge on the outer boundary
  in id order its e points, then every grid vertex on the outer boundary in
  order vy*(nx+1) + vx.

Only this module draws random numbers; the oracle and the CUDA path receive the
same arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

OP_POISSON = 0
OP_DIFFUSION = 1
OP_BIHARMONIC = 2


@dataclasses.dataclass
class Problem:
    nx: int
    ny: int
    box: tuple
    op: int
    M: np.ndarray            # [n_sub] neurons per subdomain
    w_hat: np.ndarray        # [sum M, 2]
    b_hat: np.ndarray        # [sum M]
    scale: float             # s: w = s*w_hat, b = s*b_hat
    n_int: np.ndarray        # [n_sub]
    x_int: np.ndarray        # [sum n_int, 2]
    a_int: np.ndarray        # [sum n_int]      (diffusion coefficient a at x_int)
    grad_a_int: np.ndarray   # [sum n_int, 2]   (grad a at x_int)
    edge_pts: np.ndarray     # [n_edges] points strictly inside every grid edge
    f_int: np.ndarray        # [sum n_int, R] forcing at interior points
    g_bnd: np.ndarray        # [n_bnd, R] Dirichlet data at the global boundary points
                             # (biharmonic: [2 n_bnd, R], the values of u, then of Lap u)
    n_eval: np.ndarray       # [n_sub]
    x_eval: np.ndarray       # [sum n_eval, 2]
    u_eval_exact: np.ndarray  # [sum n_eval, R] exact solution where known (else NaN)
    name: str = ""

    @property
    def n_sub(self) -> int:
        return self.nx * self.ny

    @property
    def n_rhs(self) -> int:
        return self.f_int.shape[1]


def subdomain_box(nx, ny, box, i):
    x0, x1, y0, y1 = box
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    ix, iy = i % nx, i // nx
    return x0 + ix * hx, x0 + (ix + 1) * hx, y0 + iy * hy, y0 + (iy + 1) * hy


def edge_endpoints(nx, ny, box, eid):
    """Start and end vertex (vx, vy) of grid edge eid."""
    H = nx * (ny + 1)
    if eid < H:
        vy, ix = divmod(eid, nx)
        return (ix, vy), (ix + 1, vy)
    vx, iy = divmod(eid - H, ny)
    return (vx, iy), (vx, iy + 1)


def vertex_xy(nx, ny, box, v):
    x0, x1, y0, y1 = box
    return x0 + v[0] * (x1 - x0) / nx, y0 + v[1] * (y1 - y0) / ny


def boundary_points(nx, ny, box, edge_pts):
    """Coordinates of the global Dirichlet point list (order in the module doc)."""
    pts = []
    n_edges = nx * (ny + 1) + (nx + 1) * ny
    for eid in range(n_edges):
        a, b = edge_endpoints(nx, ny, box, eid)
        on_bnd = (a[1] == b[1] and a[1] in (0, ny)) or (a[0] == b[0] and a[0] in (0, nx))
        if not on_bnd:
            continue
        pa, pb = np.array(vertex_xy(nx, ny, box, a)), np.array(vertex_xy(nx, ny, box, b))
        e = int(edge_pts[eid])
        for k in range(1, e + 1):
            pts.append(pa + k / (e + 1) * (pb - pa))
    for vy in range(ny + 1):
        for vx in range(nx + 1):
            if vx in (0, nx) or vy in (0, ny):
                pts.append(np.array(vertex_xy(nx, ny, box, (vx, vy))))
    return np.array(pts, dtype=np.float64).reshape(-1, 2)


# ----------------------------------------------------------------------------
# manufactured solutions: (u, grad u, Lap u[, Lap^2 u]) as functions of (x, y)
# arrays; the eigenfunctions below have Lap u = -k^2 u, so Lap^2 u = k^4 u
# ----------------------------------------------------------------------------

def _sin_sin(p, q):
    k2 = (p * p + q * q) * np.pi ** 2

    def u(x, y):
        return np.sin(p * np.pi * x) * np.sin(q * np.pi * y)

    def grad(x, y):
        return (p * np.pi * np.cos(p * np.pi * x) * np.sin(q * np.pi * y),
                q * np.pi * np.sin(p * np.pi * x) * np.cos(q * np.pi * y))

    def lap(x, y):
        return -k2 * u(x, y)

    def bilap(x, y):
        return k2 * k2 * u(x, y)
    return u, grad, lap, bilap


def _sin2pix_cos3piy():
    def u(x, y):
        return np.sin(2 * np.pi * x) * np.cos(3 * np.pi * y)

    def grad(x, y):
        return (2 * np.pi * np.cos(2 * np.pi * x) * np.cos(3 * np.pi * y),
                -3 * np.pi * np.sin(2 * np.pi * x) * np.sin(3 * np.pi * y))

    def lap(x, y):
        return -13 * np.pi ** 2 * u(x, y)

    def bilap(x, y):
        return 169 * np.pi ** 4 * u(x, y)
    return u, grad, lap, bilap


def coef_a(x, y):
    """a = 1 + 0.5 sin(2 pi x) sin(2 pi y) and its gradient."""
    a = 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    ax = np.pi * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    ay = np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    return a, ax, ay


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------

def make_problem(nx, ny, M, n_int, edge_pts, *, scale, init, seed, solutions,
                 op=OP_POISSON, box=(0.0, 1.0, 0.0, 1.0), n_eval=32,
                 forcing=None, coef=None, exact_known=True, points="random", name=""):
    """Draw one problem.

    M, n_int: int or per-subdomain arrays.  edge_pts: int or per-edge array.
    init: "uniform" (w_hat, b_hat ~ U[-1, 1]) or "paper" (w_hat ~ U[-1,1]^2,
    b_hat = -w_hat . xi with xi uniform in the subdomain's box enlarged by
    r = diam/2 on every side, so that b = -w . xi as in Sec. 4.1).
    solutions: list of (u, grad u, lap u[, bilap u]) tuples, one per right-hand
    side (the biharmonic operator, op 2, needs bilap: f = Lap^2 u, and the
    boundary data are u, then Lap u); forcing (optional): list of f(x, y)
    callables overriding L u, with the boundary data of u all the same.  coef (optional, diffusion): (x, y) -> (a, a_x, a_y)
    in place of coef_a.  exact_known = False: u_eval_exact is NaN (no closed form).
    points = "grid": the interior points of a subdomain are the centres of a
    uniform n x n grid of cells (n_int = n^2) instead of uniform random points.
    """
    rng = np.random.default_rng(seed)
    n_sub = nx * ny
    Ms = np.broadcast_to(np.asarray(M, dtype=np.int64), (n_sub,)).copy()
    nIs = np.broadcast_to(np.asarray(n_int, dtype=np.int64), (n_sub,)).copy()
    n_edges = nx * (ny + 1) + (nx + 1) * ny
    eps = np.broadcast_to(np.asarray(edge_pts, dtype=np.int64), (n_edges,)).copy()
    w_hat, b_hat, x_int, x_ev = [], [], [], []
    for i in range(n_sub):
        xa, xb, ya, yb = subdomain_box(nx, ny, box, i)
        m = int(Ms[i])
        wh = rng.uniform(-1.0, 1.0, size=(m, 2))
        if init == "uniform":
            bh = rng.uniform(-1.0, 1.0, size=m)
        elif init == "paper":
            r = 0.5 * math.hypot(xb - xa, yb - ya)
            xi = np.stack([rng.uniform(xa - r, xb + r, m), rng.uniform(ya - r, yb + r, m)], 1)
            bh = -(wh * xi).sum(1)
        else:
            raise ValueError(init)
        w_hat.append(wh)
        b_hat.append(bh)
        nI = int(nIs[i])
        if points == "grid":
            n = int(round(np.sqrt(nI)))
            if n * n != nI:
                raise ValueError("grid points need a square n_int")
            cx = xa + (np.arange(n) + 0.5) * (xb - xa) / n
            cy = ya + (np.arange(n) + 0.5) * (yb - ya) / n
            gx, gy = np.meshgrid(cx, cy)
            x_int.append(np.stack([gx.ravel(), gy.ravel()], 1))
        else:
            x_int.append(np.stack([rng.uniform(xa, xb, nI), rng.uniform(ya, yb, nI)], 1))
        x_ev.append(np.stack([rng.uniform(xa, xb, n_eval), rng.uniform(ya, yb, n_eval)], 1))
    x_int = np.concatenate(x_int)
    x_ev = np.concatenate(x_ev)
    xb_pts = boundary_points(nx, ny, box, eps)
    if op == OP_DIFFUSION:
        a, ax, ay = (coef or coef_a)(x_int[:, 0], x_int[:, 1])
        grad_a = np.stack([ax, ay], 1)
    else:
        a, grad_a = np.ones(len(x_int)), np.zeros((len(x_int), 2))
    f_cols, g_cols, u_cols = [], [], []
    for k, sol in enumerate(solutions):
        u, gu, lu = sol[:3]
        X, Y = x_int[:, 0], x_int[:, 1]
        if forcing is not None:
            f = forcing[k](X, Y)
        elif op == OP_BIHARMONIC:
            f = sol[3](X, Y)
        elif op == OP_DIFFUSION:
            ux, uy = gu(X, Y)
            f = -a * lu(X, Y) - grad_a[:, 0] * ux - grad_a[:, 1] * uy
        else:
            f = -lu(X, Y)
        f_cols.append(f)
        g = u(xb_pts[:, 0], xb_pts[:, 1])
        if op == OP_BIHARMONIC:
            g = np.concatenate([g, lu(xb_pts[:, 0], xb_pts[:, 1])])
        g_cols.append(g)
        u_cols.append(u(x_ev[:, 0], x_ev[:, 1]) if exact_known else np.full(len(x_ev), np.nan))
    return Problem(nx=nx, ny=ny, box=tuple(float(v) for v in box), op=op, M=Ms,
                   w_hat=np.concatenate(w_hat), b_hat=np.concatenate(b_hat),
                   scale=float(scale), n_int=nIs, x_int=x_int, a_int=np.asarray(a, np.float64),
                   grad_a_int=np.asarray(grad_a, np.float64), edge_pts=eps,
                   f_int=np.stack(f_cols, 1), g_bnd=np.stack(g_cols, 1),
                   n_eval=np.full(n_sub, n_eval, np.int64), x_eval=x_ev,
                   u_eval_exact=np.stack(u_cols, 1), name=name)


def grf(alpha, seed, n_terms=256):
    """An approximate Gaussian random field (Sec. 4.3, Eq. (grf)):
    sum_{i <= n_terms} a_i sin(w_i . x + b_i) with a_i ~ N(0, alpha^4 / 256),
    w_i ~ N(0, alpha^2 I), b_i ~ U(0, 2 pi); returns (field, gradient) callables."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, alpha * alpha / 16.0, n_terms)
    w = rng.normal(0.0, alpha, (n_terms, 2))
    b = rng.uniform(0.0, 2.0 * np.pi, n_terms)

    def phase(x, y):
        return np.outer(np.ravel(x), w[:, 0]) + np.outer(np.ravel(y), w[:, 1]) + b[None, :]

    def field(x, y):
        out = np.empty(np.size(x))
        for c in range(0, np.size(x), 8192):
            out[c:c + 8192] = np.sin(phase(np.ravel(x)[c:c + 8192], np.ravel(y)[c:c + 8192])) @ a
        return out.reshape(np.shape(x))

    def grad(x, y):
        gx, gy = np.empty(np.size(x)), np.empty(np.size(x))
        for c in range(0, np.size(x), 8192):
            cs = np.cos(phase(np.ravel(x)[c:c + 8192], np.ravel(y)[c:c + 8192])) * a[None, :]
            gx[c:c + 8192] = cs @ w[:, 0]
            gy[c:c + 8192] = cs @ w[:, 1]
        return gx.reshape(np.shape(x)), gy.reshape(np.shape(x))
    return field, grad


def grf_coefficient(alpha, seed):
    """rho = tanh(grf) + 1.1 (Sec. 4.4) and its gradient (1 - tanh^2(grf)) grad grf."""
    field, grad = grf(alpha, seed)

    def coef(x, y):
        g = field(x, y)
        gx, gy = grad(x, y)
        t = np.tanh(g)
        return t + 1.1, (1.0 - t * t) * gx, (1.0 - t * t) * gy
    return coef


def _zero_solution():
    def u(x, y):
        return np.zeros(np.shape(x))

    def grad(x, y):
        return np.zeros(np.shape(x)), np.zeros(np.shape(x))

    def lap(x, y):
        return np.zeros(np.shape(x))
    return u, grad, lap


def fourier_forcing(coeffs):
    """f = sum_{p,q=1..4} a_pq sin(p pi x) sin(q pi y) and its exact Poisson solution."""
    coeffs = np.asarray(coeffs, np.float64).reshape(4, 4)

    def u(x, y):
        s = 0.0
        for p in range(4):
            for q in range(4):
                s = s + coeffs[p, q] / (np.pi ** 2 * ((p + 1) ** 2 + (q + 1) ** 2)) * \
                    np.sin((p + 1) * np.pi * x) * np.sin((q + 1) * np.pi * y)
        return s

    def grad(x, y):
        gx, gy = 0.0, 0.0
        for p in range(4):
            for q in range(4):
                c = coeffs[p, q] / (np.pi ** 2 * ((p + 1) ** 2 + (q + 1) ** 2))
                gx = gx + c * (p + 1) * np.pi * np.cos((p + 1) * np.pi * x) * np.sin((q + 1) * np.pi * y)
                gy = gy + c * (q + 1) * np.pi * np.sin((p + 1) * np.pi * x) * np.cos((q + 1) * np.pi * y)
        return gx, gy

    def lap(x, y):
        s = 0.0
        for p in range(4):
            for q in range(4):
                s = s - coeffs[p, q] * np.sin((p + 1) * np.pi * x) * np.sin((q + 1) * np.pi * y)
        return s
    return u, grad, lap


def config(name: str) -> Problem:
    """The five synthetic workloads, by name (sizes in the docstrings of each)."""
    if name == "poisson_2x2_m100":          # 2x2, M=100, 400 interior, 20 per edge, scale 2
        return make_problem(2, 2, 100, 400, 20, scale=2.0, init="uniform", seed=1001,
                            solutions=[_sin_sin(1, 1)], name=name)
    if name == "poisson_8x8_m400":          # 8x8, M=400, 1600 interior, 40 per edge, l=32
        return make_problem(8, 8, 400, 1600, 40, scale=32.0, init="paper", seed=1002,
                            solutions=[_sin2pix_cos3piy()], name=name)
    if name == "poisson_16x16_uneven":      # 16x16, M~U{200..800}, n_I=round(U[1.5,3] M), e~U{20..60}
        rng = np.random.default_rng(10030)
        M = rng.integers(200, 801, size=256)
        nI = np.round(rng.uniform(1.5, 3.0, size=256) * M).astype(np.int64)
        e = rng.integers(20, 61, size=16 * 17 * 2)
        return make_problem(16, 16, M, nI, e, scale=32.0, init="paper", seed=1003,
                            solutions=[_sin_sin(1, 1)], name=name)
    if name == "poisson_8x8_fourier":       # as 8x8 M=400 with 16-mode Fourier forcing, g=0
        rng = np.random.default_rng(10040)
        coeffs = rng.standard_normal(16)
        return make_problem(8, 8, 400, 1600, 40, scale=32.0, init="paper", seed=1004,
                            solutions=[fourier_forcing(coeffs)], name=name)
    if name == "diffusion_32x32_m1000_r16":  # 32x32, M=1000, 4000 interior, 40 per edge, 16 RHS
        sols = [_sin_sin(p, q) for p in range(1, 5) for q in range(1, 5)]
        return make_problem(32, 32, 1000, 4000, 40, scale=32.0, init="paper", seed=1005,
                            solutions=sols, op=OP_DIFFUSION, name=name)
    if name == "poisson_8x8_grf":           # the 8x8 M=400 shape, g = 0, f = GRF with alpha = 32 (Sec. 4.3)
        f, _ = grf(32.0, 1007)
        return make_problem(8, 8, 400, 1600, 40, scale=32.0, init="paper", seed=1007,
                            solutions=[_zero_solution()], forcing=[f], exact_known=False, name=name)
    if name == "varcoef_8x8_grf":           # -div(rho grad u) = 1, u = 0 on the boundary, rho = tanh(GRF) + 1.1 (Sec. 4.4)
        return make_problem(8, 8, 400, 1600, 40, scale=32.0, init="paper", seed=1008,
                            solutions=[_zero_solution()], forcing=[lambda x, y: np.ones(np.shape(x))],
                            op=OP_DIFFUSION, coef=grf_coefficient(32.0, 1009), exact_known=False, name=name)
    if name == "poisson_4x4_m400":          # the 8x8 M=400 workload's per-subdomain shape on a 4x4 grid (profiling)
        return make_problem(4, 4, 400, 1600, 40, scale=32.0, init="paper", seed=1010,
                            solutions=[_sin2pix_cos3piy()], name=name)
    if name == "poisson_8x8_m100":          # the 8x8 M=400 workload's interface (40 per edge) with M=100, 400 interior (profiling the CG)
        return make_problem(8, 8, 100, 400, 40, scale=32.0, init="paper", seed=1011,
                            solutions=[_sin2pix_cos3piy()], name=name)
    if name == "biharmonic_16x16":          # Sec. 4.5 at 16x16: M=256, 20x20 grid, 20 per edge, l=64
        return paper_scale(16, op=OP_BIHARMONIC)
    if name == "diffusion_4x4_m1000_r16":   # the 32x32 workload's per-subdomain shape on a 4x4 grid
        sols = [_sin_sin(p, q) for p in range(1, 5) for q in range(1, 5)]
        return make_problem(4, 4, 1000, 4000, 40, scale=32.0, init="paper", seed=1006,
                            solutions=sols, op=OP_DIFFUSION, name=name)
    raise KeyError(name)


CONFIGS = ("poisson_2x2_m100", "poisson_8x8_m400", "poisson_16x16_uneven",
           "poisson_8x8_fourier", "diffusion_32x32_m1000_r16")


def interface_vectors(n_delta, n_rhs, count, seed):
    """`count` seeded N(0, 1) interface vectors [n_delta x n_rhs] (inputs of the
    operator-application checks)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((n_delta, n_rhs)) for _ in range(count)]


def fourier_basis(x):
    """sin(p pi x) sin(q pi y), p, q = 1..4, at the points x [n x 2] -> [n x 16]
    (column 4 (p-1) + (q-1)), the modes of the Fourier forcing."""
    return np.stack([np.sin(p * np.pi * x[:, 0]) * np.sin(q * np.pi * x[:, 1])
                     for p in range(1, 5) for q in range(1, 5)], 1)


def fourier_coefficients():
    """The 16 coefficients a_pq of the poisson_8x8_fourier forcing (row p-1, column q-1 flattened)."""
    return np.random.default_rng(10040).standard_normal(16)


def paper_scale(n, seed=2001, max_neurons=1024, op=OP_POISSON):
    """The paper's setting (Sec. 4.1, Sec. 4.2, Sec. 4.5): n x n subdomains of
    the unit square, 2^16 neurons in total (2^16 / n^2 per subdomain, capped at
    max_neurons, the library's per-subdomain limit), a (320 / n) x (320 / n)
    uniform grid per subdomain (cell centres inside, 320 / n points on every
    edge), the paper's initialisation with l = 32 (Poisson) or l = 64
    (biharmonic), u = sin(pi x) sin(pi y)."""
    g = 320 // n
    M = min(2 ** 16 // (n * n), max_neurons)
    scale = 64.0 if op == OP_BIHARMONIC else 32.0
    tag = "biharmonic" if op == OP_BIHARMONIC else "paper"
    return make_problem(n, n, M, g * g, g, scale=scale, init="paper", seed=seed, solutions=[_sin_sin(1, 1)],
                        points="grid", op=op, name=f"{tag}_{n}x{n}")


def small_uneven_problem(nx=4, ny=3, M_range=(20, 90), seed=13, n_rhs=1, init="paper", scale=8.0):
    """Small problem with uneven subdomains: neurons, interior points (1.5-3 x M)
    and points per edge all drawn per subdomain / per edge."""
    rng = np.random.default_rng(seed)
    n_sub = nx * ny
    M = rng.integers(M_range[0], M_range[1] + 1, size=n_sub)
    nI = np.round(rng.uniform(1.5, 3.0, size=n_sub) * M).astype(np.int64)
    e = rng.integers(2, 7, size=nx * (ny + 1) + (nx + 1) * ny)
    sols = [_sin_sin(1, 1), _sin2pix_cos3piy(), _sin_sin(2, 1), _sin_sin(1, 3)][:n_rhs]
    return make_problem(nx, ny, M, nI, e, scale=scale, init=init, seed=seed + 1, solutions=sols,
                        n_eval=8, name="small_uneven")


def small_problem(nx=2, ny=2, M=12, n_int=40, edge_pts=3, *, seed=7, scale=3.0,
                  init="uniform", n_rhs=1, op=OP_POISSON, n_eval=8):
    """Tiny problems for brute-force checks (any grid, any sizes)."""
    sols = [_sin_sin(1, 1), _sin2pix_cos3piy(), _sin_sin(2, 1), _sin_sin(1, 3)][:n_rhs]
    while len(sols) < n_rhs:
        sols.append(_sin_sin(len(sols) % 4 + 1, len(sols) // 4 + 1))
    return make_problem(nx, ny, M, n_int, edge_pts, scale=scale, init=init, seed=seed,
                        solutions=sols, op=op, n_eval=n_eval, name="small")
