"""Decomposition layout for the oracle (test infrastructure only).

Follows the point sets of Sec. 2.2.1 (x_I, x_B, x_Gamma per subdomain), the
split Gamma = Pi u Delta of Sec. 3 (Pi = interior cross points of the grid of
subdomains), the change of variables T^i of Sec. 3.2 (Fig. "change": the
coarse variable of a cross point is the linear function along each incident
edge, so a Delta point at arc fraction s from the edge start carries weight
1-s on the start vertex and s on the end vertex, each only if that vertex is in
Pi), and the modified flux A_m of Sec. 3.2 (the row of a cross point p is the
mean flux over the points of an incident edge, opposite end excluded, summed
over the edges of the subdomain that meet p).

Geometry conventions (independent restatement of the problem format):
subdomain (ix, iy) = index iy*nx+ix; horizontal edge (ix, vy) has id vy*nx+ix,
vertical edge (vx, iy) has id nx*(ny+1)+vx*ny+iy; edge points at
start + k/(e+1)(end-start), k=1..e; global Dirichlet list = boundary-edge
points in edge order, then boundary vertices in order vy*(nx+1)+vx; global
Gamma = Pi (cross points in order (vy-1)*(nx-1)+(vx-1)) then Delta (interface
edges in id order, points k=1..e).
"""
from __future__ import annotations

import numpy as np


class SubLayout:
    """Per-subdomain point sets and index maps."""

    def __init__(self):
        self.bnd_xy = None        # [nB, 2]
        self.bnd_gidx = None      # [nB] index into the global Dirichlet list
        self.pi_xy = None         # [nPi, 2] local cross points (BL, BR, TL, TR order)
        self.pi_gidx = None       # [nPi] global Pi index
        self.pi_vertex = None     # list of (vx, vy)
        self.dl_xy = None         # [nDl, 2] local Delta points
        self.dl_gidx = None       # [nDl] global Gamma index (>= n_Pi)
        self.dl_normal = None     # [nDl, 2] outward normal of this subdomain
        self.dl_alpha = None      # [nDl] T weight on the start vertex
        self.dl_alpha_pi = None   # [nDl] local Pi index of the start vertex or -1
        self.dl_beta = None       # [nDl] T weight on the end vertex
        self.dl_beta_pi = None    # [nDl] local Pi index of the end vertex or -1
        self.am_terms = None      # per local Pi: list of (weight, xy, normal)
        # interface / boundary component of every row: 0 the value and the normal
        # derivative of u; 1 (biharmonic) those of Lap u
        self.bnd_comp = None
        self.pi_comp = None
        self.dl_comp = None


class Layout:
    def __init__(self, nx, ny, box, edge_pts, use_Am=True, n_comp=1, use_coarse=True):
        """use_Am: the corner rows of A_m (Sec. 3.2); False: the plain flux rows
        of Eq. (ddelm), whose corner row (the corner normal is undefined) is the
        sum over the two edges of the subdomain meeting the corner of the flux
        there with that edge's normal.

        n_comp = 2 (the biharmonic coupled system of Sec. 2.1: u and Lap u are
        both continuous across the interface, and both normal derivatives
        balance): every boundary, Pi and Delta point carries two rows.  Global
        numbering: the Dirichlet list holds the u data, then the Lap u data;
        Gamma = Pi (component 0, then 1), then Delta (component 0, then 1); in a
        subdomain the rows of component 1 follow those of component 0 in each
        block, and its change of variables and A_m rows combine rows of the
        same component.

        use_coarse = False: vanilla DDELM (Sec. 2.2.1, Eq. (schur)), no coarse
        space: Pi is empty and every cross point is an interface point of the
        Delta set shared by its four subdomains, numbered before the edge
        points (in cross-point order).  Its flux row in subdomain i is the plain
        one of Eq. (ddelm) with the undefined corner normal resolved as in the
        plain-A reading above: the sum of the outward normals of the two edges
        of subdomain i that meet there (the flux is linear in the normal)."""
        self.use_Am = use_Am
        self.n_comp = n_comp
        self.use_coarse = use_coarse
        self.nx, self.ny, self.box = nx, ny, box
        self.edge_pts = np.asarray(edge_pts, np.int64)
        x0, x1, y0, y1 = box
        self.hx, self.hy = (x1 - x0) / nx, (y1 - y0) / ny
        H = nx * (ny + 1)
        self.n_edges = H + (nx + 1) * ny
        # global Dirichlet list
        bnd_off = {}
        nb = 0
        for eid in range(self.n_edges):
            if self.edge_on_boundary(eid):
                bnd_off[eid] = nb
                nb += int(self.edge_pts[eid])
        vtx_bnd = {}
        for vy in range(ny + 1):
            for vx in range(nx + 1):
                if vx in (0, nx) or vy in (0, ny):
                    vtx_bnd[(vx, vy)] = nb
                    nb += 1
        self.n_bnd = nb
        # global Gamma
        n_cross = (nx - 1) * (ny - 1)
        self.n_pi = n_cross if use_coarse else 0
        dl_off = {}
        nd = 0 if use_coarse else n_cross      # vanilla: the cross points open the Delta list
        for eid in range(self.n_edges):
            if not self.edge_on_boundary(eid):
                dl_off[eid] = self.n_pi + nd
                nd += int(self.edge_pts[eid])
        self.n_delta = nd
        self.n_gamma = self.n_pi + nd
        self.subs = []
        for i in range(nx * ny):
            self.subs.append(self._sub(i, bnd_off, vtx_bnd, dl_off))
        if n_comp == 2:
            self._second_component()
        elif n_comp != 1:
            raise ValueError("n_comp must be 1 or 2")

    def _second_component(self):
        nb, npi, nd = self.n_bnd, self.n_pi, self.n_delta
        for s in self.subs:
            kb, kp, kd = len(s.bnd_xy), len(s.pi_xy), len(s.dl_xy)
            s.bnd_xy = np.vstack([s.bnd_xy, s.bnd_xy])
            s.bnd_gidx = np.concatenate([s.bnd_gidx, s.bnd_gidx + nb])
            s.bnd_comp = np.repeat([0, 1], kb)
            s.pi_xy = np.vstack([s.pi_xy, s.pi_xy])
            s.pi_gidx = np.concatenate([s.pi_gidx, s.pi_gidx + npi])
            s.pi_vertex = s.pi_vertex + s.pi_vertex
            s.pi_comp = np.repeat([0, 1], kp)
            d0 = s.dl_gidx - npi                      # Delta position of component 0
            s.dl_xy = np.vstack([s.dl_xy, s.dl_xy])
            s.dl_gidx = np.concatenate([2 * npi + d0, 2 * npi + nd + d0])
            s.dl_normal = np.vstack([s.dl_normal, s.dl_normal])
            s.dl_comp = np.repeat([0, 1], kd)
            s.dl_alpha = np.concatenate([s.dl_alpha, s.dl_alpha])
            s.dl_beta = np.concatenate([s.dl_beta, s.dl_beta])
            s.dl_alpha_pi = np.concatenate([s.dl_alpha_pi, np.where(s.dl_alpha_pi >= 0, s.dl_alpha_pi + kp, -1)])
            s.dl_beta_pi = np.concatenate([s.dl_beta_pi, np.where(s.dl_beta_pi >= 0, s.dl_beta_pi + kp, -1)])
            s.am_terms = s.am_terms + s.am_terms
        self.n_bnd, self.n_pi, self.n_delta = 2 * nb, 2 * npi, 2 * nd
        self.n_gamma = self.n_pi + self.n_delta

    # ------------------------------------------------------------------
    def edge_on_boundary(self, eid):
        nx, ny = self.nx, self.ny
        H = nx * (ny + 1)
        if eid < H:
            vy = eid // nx
            return vy == 0 or vy == ny
        vx = (eid - H) // ny
        return vx == 0 or vx == nx

    def is_cross(self, v):
        return 0 < v[0] < self.nx and 0 < v[1] < self.ny

    def pi_index(self, v):
        return (v[1] - 1) * (self.nx - 1) + (v[0] - 1)

    def vxy(self, v):
        return np.array([self.box[0] + v[0] * self.hx, self.box[2] + v[1] * self.hy])

    def _sub(self, i, bnd_off, vtx_bnd, dl_off):
        nx, ny = self.nx, self.ny
        H = nx * (ny + 1)
        ix, iy = i % nx, i // nx
        BL, BR, TL, TR = (ix, iy), (ix + 1, iy), (ix, iy + 1), (ix + 1, iy + 1)
        # (edge id, start vertex, end vertex, outward normal)
        edges = [(iy * nx + ix, BL, BR, (0.0, -1.0)),
                 ((iy + 1) * nx + ix, TL, TR, (0.0, 1.0)),
                 (H + ix * ny + iy, BL, TL, (-1.0, 0.0)),
                 (H + (ix + 1) * ny + iy, BR, TR, (1.0, 0.0))]
        s = SubLayout()
        bxy, bg = [], []
        for eid, a, b, _ in edges:
            if self.edge_on_boundary(eid):
                e = int(self.edge_pts[eid])
                pa, pb = self.vxy(a), self.vxy(b)
                for k in range(1, e + 1):
                    bxy.append(pa + k / (e + 1) * (pb - pa))
                    bg.append(bnd_off[eid] + k - 1)
        for v in (BL, BR, TL, TR):
            if not self.is_cross(v) and (v[0] in (0, nx) or v[1] in (0, ny)):
                bxy.append(self.vxy(v))
                bg.append(vtx_bnd[v])
        s.bnd_xy = np.array(bxy).reshape(-1, 2)
        s.bnd_gidx = np.array(bg, np.int64)
        crosses = [v for v in (BL, BR, TL, TR) if self.is_cross(v)]
        pis = crosses if self.use_coarse else []
        s.pi_vertex = pis
        s.pi_xy = np.array([self.vxy(v) for v in pis]).reshape(-1, 2)
        s.pi_gidx = np.array([self.pi_index(v) for v in pis], np.int64)
        loc_pi = {v: k for k, v in enumerate(pis)}
        dxy, dg, dn, al, alp, be, bep = [], [], [], [], [], [], []
        if not self.use_coarse:
            for v in crosses:
                nsum = np.zeros(2)
                for eid, a, b, nrm in edges:
                    if v in (a, b):
                        nsum += nrm
                dxy.append(self.vxy(v))
                dg.append(self.pi_index(v))          # Delta index = cross-point order
                dn.append(nsum)
                al.append(0.0)
                alp.append(-1)
                be.append(0.0)
                bep.append(-1)
        for eid, a, b, nrm in edges:
            if self.edge_on_boundary(eid):
                continue
            e = int(self.edge_pts[eid])
            pa, pb = self.vxy(a), self.vxy(b)
            for k in range(1, e + 1):
                frac = k / (e + 1)
                dxy.append(pa + frac * (pb - pa))
                dg.append(dl_off[eid] + k - 1)
                dn.append(nrm)
                al.append(1.0 - frac if a in loc_pi else 0.0)
                alp.append(loc_pi.get(a, -1))
                be.append(frac if b in loc_pi else 0.0)
                bep.append(loc_pi.get(b, -1))
        s.dl_xy = np.array(dxy).reshape(-1, 2)
        s.dl_gidx = np.array(dg, np.int64)
        s.dl_normal = np.array(dn).reshape(-1, 2)
        s.dl_alpha, s.dl_alpha_pi = np.array(al), np.array(alp, np.int64)
        s.dl_beta, s.dl_beta_pi = np.array(be), np.array(bep, np.int64)
        # A_m rows of the cross points: mean flux over (p and the edge's e points)
        terms = []
        for v in pis:
            t = []
            for eid, a, b, nrm in edges:
                if v not in (a, b):
                    continue
                if not self.use_Am:
                    t.append((1.0, self.vxy(v), nrm))
                    continue
                e = int(self.edge_pts[eid])
                wgt = 1.0 / (e + 1)
                pa, pb = self.vxy(a), self.vxy(b)
                t.append((wgt, self.vxy(v), nrm))
                for k in range(1, e + 1):
                    t.append((wgt, pa + k / (e + 1) * (pb - pa), nrm))
            terms.append(t)
        s.am_terms = terms
        s.bnd_comp = np.zeros(len(s.bnd_xy), np.int64)
        s.pi_comp = np.zeros(len(s.pi_xy), np.int64)
        s.dl_comp = np.zeros(len(s.dl_xy), np.int64)
        return s
