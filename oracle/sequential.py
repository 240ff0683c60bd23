"""Procedures 1-4 of arxiv 1805.08500 (Sec. 3.1) restated sequentially, for
tiny scenes -- TEST INFRASTRUCTURE ONLY.

This is a second, independent algorithm used to pin the C oracle. It shares
no code with ``spm_oracle.c``:

* DataArray holds the sources (point sources, then per segment: endpoint A,
  endpoint B and its interior, Sec. 4) and every obstacle vertex.
* Each iteration picks the unexpanded entry with the smallest Distance
  (Procedure 1, "Search"), then for every pixel that sees it sets
  newDist = Distance + |p - g| when smaller (Procedure 3, "Cone"), and does the
  same for every obstacle vertex (Procedure 4, "Distance"). A segment interior
  reaches a point through its perpendicular foot when the foot falls strictly
  inside the segment (the Sec. 4 distance rule); otherwise the endpoints,
  which are ordinary sources, cover it.
* Visibility is exact and uses a different method from the C oracle: every
  parameter where the segment touches an obstacle boundary is found with
  rational arithmetic, and the segment is blocked iff the midpoint of some
  piece between consecutive contacts lies strictly inside the obstacle.
* No cone restriction (the paper has none), so labels may differ from the C
  oracle only where two generators tie exactly.

Only scenes of pairwise disjoint convex polygons are supported (every vertex
is then a corner of free space).
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np


def lattice_scale(world, grid, polys) -> int:
    Wx, Wy = world
    Nx, Ny = grid
    S = 1
    while (S * Wx) % (2 * Nx) or (S * Wy) % (2 * Ny):
        S *= 2
    xs = [0, Wx] + [int(v) for p in polys for v in p[:, 0]]
    ys = [0, Wy] + [int(v) for p in polys for v in p[:, 1]]
    span = max(max(xs) - min(xs), max(ys) - min(ys))
    assert S * span <= 32767
    while 2 * S * span <= 32767:
        S *= 2
    return S


def _orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


class Sequential:
    def __init__(self, scene):
        self.scene = scene
        S = self.S = lattice_scale(scene.world, scene.grid, scene.polys)
        self.polys = []
        for p in scene.polys:
            pts = [(int(x) * S, int(y) * S) for x, y in p]
            area2 = sum(pts[i][0] * pts[(i + 1) % len(pts)][1]
                        - pts[(i + 1) % len(pts)][0] * pts[i][1] for i in range(len(pts)))
            if area2 < 0:
                pts = pts[::-1]
            self.polys.append(pts)
        self.bbox = [(min(x for x, _ in P), min(y for _, y in P), max(x for x, _ in P),
                      max(y for _, y in P)) for P in self.polys]
        # DataArray entries: (kind, lattice xy, true xy, segment index)
        ent = []
        for (x, y) in scene.points:
            ent.append(("point", (round(x * S), round(y * S)), (float(x), float(y)), -1))
        for k, (ax, ay, bx, by) in enumerate(scene.segs):
            A = (round(ax * S), round(ay * S))
            B = (round(bx * S), round(by * S))
            ent.append(("point", A, (float(ax), float(ay)), k))
            ent.append(("point", B, (float(bx), float(by)), k))
            ent.append(("segment", A, (float(ax), float(ay)), k))
        self.n_src = len(ent)
        for P in self.polys:
            for v in P:
                ent.append(("vertex", v, (v[0] / S, v[1] / S), -1))
        self.ent = ent
        self.seg_lat = [((round(ax * S), round(ay * S)), (round(bx * S), round(by * S)))
                        for (ax, ay, bx, by) in scene.segs]

    # ------------------------------------------------------------------
    def _blocked(self, p, q) -> bool:
        """Open segment p->q (rational points) meets some open interior?"""
        if p == q:
            return False
        lo_x, hi_x = min(p[0], q[0]), max(p[0], q[0])
        lo_y, hi_y = min(p[1], q[1]), max(p[1], q[1])
        dx, dy = q[0] - p[0], q[1] - p[1]
        for P, (bx0, by0, bx1, by1) in zip(self.polys, self.bbox):
            if bx1 < lo_x or bx0 > hi_x or by1 < lo_y or by0 > hi_y:
                continue
            ts = {Fr(0), Fr(1)}
            m = len(P)
            for i in range(m):
                a, b = P[i], P[(i + 1) % m]
                ex, ey = b[0] - a[0], b[1] - a[1]
                den = dx * ey - dy * ex
                wx, wy = a[0] - p[0], a[1] - p[1]
                if den != 0:
                    t = Fr(wx * ey - wy * ex) / den
                    s = Fr(wx * dy - wy * dx) / den
                    if 0 <= t <= 1 and 0 <= s <= 1:
                        ts.add(t)
                elif wx * dy - wy * dx == 0:  # collinear: overlap end points
                    L2 = dx * dx + dy * dy
                    for c in (a, b):
                        t = Fr((c[0] - p[0]) * dx + (c[1] - p[1]) * dy) / L2
                        if 0 <= t <= 1:
                            ts.add(t)
            ts = sorted(ts)
            for t0, t1 in zip(ts[:-1], ts[1:]):
                tm = (t0 + t1) / 2
                mpt = (p[0] + tm * dx, p[1] + tm * dy)
                if all(_orient(P[i], P[(i + 1) % m], mpt) > 0 for i in range(m)):
                    return True
        return False

    def _foot(self, k, q):
        """Perpendicular foot of lattice point q on segment k if strictly inside."""
        A, B = self.seg_lat[k]
        ux, uy = B[0] - A[0], B[1] - A[1]
        num = (q[0] - A[0]) * ux + (q[1] - A[1]) * uy
        den = ux * ux + uy * uy
        if not (0 < num < den):
            return None
        t = Fr(num, den)
        return (A[0] + t * ux, A[1] + t * uy)

    def _reach(self, idx, q_lat, q_true):
        """Distance from DataArray entry idx to a point q, or None if not seen."""
        kind, g_lat, g_true, k = self.ent[idx]
        if kind == "segment":
            f = self._foot(k, q_lat)
            if f is None or self._blocked(q_lat, f):
                return None
            ax, ay, bx, by = (float(v) for v in self.scene.segs[k])
            ux, uy = bx - ax, by - ay
            return abs(ux * (q_true[1] - ay) - uy * (q_true[0] - ax)) / math.sqrt(ux * ux + uy * uy)
        if self._blocked(q_lat, g_lat):
            return None
        dx, dy = q_true[0] - g_true[0], q_true[1] - g_true[1]
        return math.sqrt(dx * dx + dy * dy)

    def _free(self, q):
        return not any(all(_orient(P[i], P[(i + 1) % len(P)], q) > 0 for i in range(len(P)))
                       for P in self.polys)

    def run(self):
        """Returns (dist (Ny,Nx), parent (Ny,Nx), vertex Distance, ParentId)."""
        sc = self.scene
        (Wx, Wy), (Nx, Ny) = sc.world, sc.grid
        S = self.S
        n = len(self.ent)
        dist = [0.0 if i < self.n_src else math.inf for i in range(n)]
        parent = [i if i < self.n_src else -1 for i in range(n)]
        expanded = [False] * n
        pix = []
        for j in range(Ny):
            for i in range(Nx):
                q = ((2 * i + 1) * S * Wx // (2 * Nx), (2 * j + 1) * S * Wy // (2 * Ny))
                qt = ((i + 0.5) * Wx / Nx, (j + 0.5) * Wy / Ny)
                pix.append((q, qt, self._free(q)))
        F = np.full(len(pix), math.inf)
        L = np.full(len(pix), -1, dtype=np.int64)
        for _ in range(n):
            # Procedure 1: smallest Distance among unexpanded entries
            g, best = -1, math.inf
            for i in range(n):
                if not expanded[i] and dist[i] < best:
                    g, best = i, dist[i]
            if g < 0:
                break
            expanded[g] = True
            # Procedure 3: pixels that see g
            for pi, (q, qt, free) in enumerate(pix):
                if not free:
                    continue
                r = self._reach(g, q, qt)
                if r is None:
                    continue
                nd = dist[g] + r
                if nd < F[pi]:
                    F[pi] = nd
                    L[pi] = g
            # Procedure 4: obstacle vertices that see g
            for v in range(self.n_src, n):
                if v == g:
                    continue
                r = self._reach(g, self.ent[v][1], self.ent[v][2])
                if r is None:
                    continue
                nd = dist[g] + r
                if nd < dist[v]:
                    dist[v] = nd
                    parent[v] = g
        return F.reshape(Ny, Nx), L.reshape(Ny, Nx), np.array(dist), np.array(parent)

    def visibility_matrix(self):
        """sees[u][v] for DataArray entries u (any) and obstacle vertices v."""
        n = len(self.ent)
        M = np.zeros((n, n), dtype=bool)
        for u in range(n):
            for v in range(self.n_src, n):
                if u != v and self._reach(u, self.ent[v][1], self.ent[v][2]) is not None:
                    M[u, v] = True
        return M

    def edge_length(self, u, v):
        return self._reach(u, self.ent[v][1], self.ent[v][2])
