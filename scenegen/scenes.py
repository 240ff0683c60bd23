"""Seeded scene generators (SplitMix64 -> uniforms) and a JSON scene format.

Every workload is drawn from a named, platform-independent PRNG (SplitMix64)
and uses only IEEE-exact operations (add, multiply, divide, sqrt, rounding)
so the same seed yields the same integer geometry on x86 and Arm hosts.

Scene conventions (shared by the library and the oracle as *data*):
  * world is [0, Wx) x [0, Wy) in integer world units, grid Nx x Ny pixels;
  * obstacles are convex polygons with integer vertices (any orientation);
  * point sources are (x, y) pairs, segment sources (ax, ay, bx, by);
  * the recipe of each configuration is in its generator's docstring.
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014) with 53-bit uniform doubles."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + min(int(self.uniform() * span), span - 1)

    def unit_vector(self, upper_half: bool = False):
        """Uniform direction by rejection in the unit disc (no libm calls)."""
        while True:
            u = self.uniform(-1.0, 1.0)
            v = self.uniform(0.0, 1.0) if upper_half else self.uniform(-1.0, 1.0)
            r2 = u * u + v * v
            if 0.0625 < r2 <= 1.0:
                n = math.sqrt(r2)
                return u / n, v / n

    def shuffle(self, xs: list) -> list:
        for i in range(len(xs) - 1, 0, -1):
            j = self.randint(0, i)
            xs[i], xs[j] = xs[j], xs[i]
        return xs


@dataclass
class Scene:
    world: tuple
    grid: tuple
    polys: List[np.ndarray]
    points: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    segs: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))
    name: str = "scene"
    seed: int = 0
    meta: dict = field(default_factory=dict)
    agents: Optional[np.ndarray] = None  # (n, 2) int32 pixel indices (i, j)

    def __post_init__(self):
        self.world = (int(self.world[0]), int(self.world[1]))
        self.grid = (int(self.grid[0]), int(self.grid[1]))
        self.polys = [np.asarray(p, dtype=np.int32).reshape(-1, 2) for p in self.polys]
        self.points = np.asarray(self.points, dtype=np.float64).reshape(-1, 2)
        self.segs = np.asarray(self.segs, dtype=np.float64).reshape(-1, 4)

    @property
    def n_pixels(self) -> int:
        return self.grid[0] * self.grid[1]

    def flat(self):
        """(poly_off int32[P+1], poly_xy int32[2V]) CSR arrays."""
        off = np.zeros(len(self.polys) + 1, dtype=np.int32)
        for i, p in enumerate(self.polys):
            off[i + 1] = off[i] + len(p)
        xy = (np.concatenate(self.polys).reshape(-1) if self.polys
              else np.zeros(0, np.int32)).astype(np.int32)
        return off, np.ascontiguousarray(xy)

    def to_json(self) -> dict:
        d = {
            "name": self.name, "seed": self.seed, "world": list(self.world),
            "grid": list(self.grid), "polys": [p.tolist() for p in self.polys],
            "points": self.points.tolist(), "segs": self.segs.tolist(),
            "meta": self.meta,
        }
        if self.agents is not None:
            d["agents"] = np.asarray(self.agents).tolist()
        return d

    @staticmethod
    def from_json(d: dict) -> "Scene":
        ag = d.get("agents")
        return Scene(world=tuple(d["world"]), grid=tuple(d["grid"]),
                     polys=[np.array(p, dtype=np.int32) for p in d["polys"]],
                     points=np.array(d["points"], dtype=np.float64).reshape(-1, 2),
                     segs=np.array(d["segs"], dtype=np.float64).reshape(-1, 4),
                     name=d.get("name", "scene"), seed=d.get("seed", 0),
                     meta=d.get("meta", {}),
                     agents=None if ag is None else np.array(ag, dtype=np.int32))


def save_scene(scene: Scene, path: str) -> None:
    with open(path, "w") as f:
        json.dump(scene.to_json(), f)


def load_scene(path: str) -> Scene:
    with open(path) as f:
        return Scene.from_json(json.load(f))


# ---------------------------------------------------------------------------
# helpers used only to *place* obstacles and sources (rejection sampling)
# ---------------------------------------------------------------------------

def _strict_hull(pts):
    """Strictly convex hull (collinear points dropped), counter-clockwise."""
    pts = sorted(set(pts))
    if len(pts) < 3:
        return pts

    def turn(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in pts:
        while len(lower) >= 2 and turn(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(pts):
        while len(upper) >= 2 and turn(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return lower[:-1] + upper[:-1]


def _angle_key(v):
    """Sort key equivalent to the polar angle in [0, 2pi) using exact tests."""
    x, y = v
    half = 0 if (y > 0 or (y == 0 and x > 0)) else 1
    return half, v


def _random_convex(rng: SplitMix64, cx, cy, r, k):
    dirs = [rng.unit_vector() for _ in range(k)]
    # order by polar angle: bucket by half-plane, then by cross product
    import functools

    def cmp(a, b):
        ha, hb = _angle_key(a)[0], _angle_key(b)[0]
        if ha != hb:
            return ha - hb
        c = a[0] * b[1] - a[1] * b[0]
        return -1 if c > 0 else (1 if c < 0 else 0)

    dirs.sort(key=functools.cmp_to_key(cmp))
    pts = [(int(round(cx + r * dx)), int(round(cy + r * dy))) for dx, dy in dirs]
    return _strict_hull(pts)


def _place_convex_polys(rng, W, n, r_lo=20.0, r_hi=120.0, k_lo=4, k_hi=8,
                        max_attempts=1000):
    """Rejection-place n convex polygons whose bounding circles (radius r+1)
    are pairwise >= 1 unit apart and >= 1 unit inside the world."""
    circles, polys = [], []
    for _ in range(n):
        for _attempt in range(max_attempts):
            r = rng.uniform(r_lo, r_hi)
            k = rng.randint(k_lo, k_hi)
            rb = r + 1.0
            lo, hi = rb + 1.0, W - rb - 1.0
            if hi <= lo:
                continue
            cx = rng.uniform(lo, hi)
            cy = rng.uniform(lo, hi)
            ok = True
            for (ox, oy, orb) in circles:
                dx, dy = cx - ox, cy - oy
                if dx * dx + dy * dy < (rb + orb + 1.0) ** 2:
                    ok = False
                    break
            if not ok:
                continue
            hull = _random_convex(rng, cx, cy, r, k)
            if len(hull) < 3:
                continue
            circles.append((cx, cy, rb))
            polys.append(np.array(hull, dtype=np.int32))
            break
    return polys, circles


def _free_of_circles(x, y, circles, margin=1.0):
    for (ox, oy, orb) in circles:
        dx, dy = x - ox, y - oy
        if dx * dx + dy * dy <= (orb + margin) ** 2:
            return False
    return True


def _seg_clear_of_circles(ax, ay, bx, by, circles, margin=1.0):
    """True when the closed segment stays > margin outside every circle."""
    ux, uy = bx - ax, by - ay
    L2 = ux * ux + uy * uy
    for (ox, oy, orb) in circles:
        t = ((ox - ax) * ux + (oy - ay) * uy) / L2 if L2 > 0 else 0.0
        t = min(1.0, max(0.0, t))
        qx, qy = ax + t * ux - ox, ay + t * uy - oy
        if qx * qx + qy * qy <= (orb + margin) ** 2:
            return False
    return True


def _random_point_source(rng, W, circles, integer=True):
    while True:
        if integer:
            x, y = float(rng.randint(1, W - 1)), float(rng.randint(1, W - 1))
        else:
            x = float(np.float32(rng.uniform(1.0, W - 1.0)))
            y = float(np.float32(rng.uniform(1.0, W - 1.0)))
        if _free_of_circles(x, y, circles):
            return x, y


def _random_segment_source(rng, W, circles, integer=True, len_lo=50.0, len_hi=400.0):
    while True:
        mx, my = rng.uniform(1.0, W - 1.0), rng.uniform(1.0, W - 1.0)
        L = rng.uniform(len_lo, len_hi)
        dx, dy = rng.unit_vector(upper_half=True)
        ax, ay = mx - 0.5 * L * dx, my - 0.5 * L * dy
        bx, by = mx + 0.5 * L * dx, my + 0.5 * L * dy
        if integer:
            ax, ay, bx, by = (float(round(v)) for v in (ax, ay, bx, by))
        else:
            ax, ay, bx, by = (float(np.float32(v)) for v in (ax, ay, bx, by))
        if min(ax, ay, bx, by) < 1.0 or max(ax, ay, bx, by) > W - 1.0:
            continue
        if ax == bx and ay == by:
            continue
        if _seg_clear_of_circles(ax, ay, bx, by, circles):
            return ax, ay, bx, by


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def plain_rects(seed: int = 0, W: int = 256, N: int = 256, n_rects: int = 8,
                side=(8, 40), n_points: int = 1) -> Scene:
    """256^2 grid over [0,256)^2: 8 axis-aligned rectangles, sides uniform
    8..40 (integer), rejection-placed >= 1 unit apart and >= 1 unit inside the
    world; one point source at a uniform integer position outside every
    closed rectangle."""
    rng = SplitMix64(seed * 0x1000193 + 11)
    rects = []
    while len(rects) < n_rects:
        for _ in range(1000):
            w, h = rng.randint(*side), rng.randint(*side)
            x0, y0 = rng.randint(1, W - 1 - w), rng.randint(1, W - 1 - h)
            x1, y1 = x0 + w, y0 + h
            if all(x0 >= b[2] + 1 or x1 <= b[0] - 1 or y0 >= b[3] + 1 or y1 <= b[1] - 1
                   for b in rects):
                rects.append((x0, y0, x1, y1))
                break
        else:
            break
    pts = []
    while len(pts) < n_points:
        x, y = rng.randint(0, W - 1), rng.randint(0, W - 1)
        if all(not (b[0] <= x <= b[2] and b[1] <= y <= b[3]) for b in rects):
            pts.append((float(x), float(y)))
    polys = [np.array([(b[0], b[1]), (b[2], b[1]), (b[2], b[3]), (b[0], b[3])], np.int32)
             for b in rects]
    return Scene((W, W), (N, N), polys, np.array(pts), np.zeros((0, 4)),
                 name=f"plain_rects_{N}", seed=seed,
                 meta={"n_rects": len(rects)})


def plain_polys(seed: int = 0, W: int = 4096, N: int = 1024, n_polys: int = 200,
                n_points: int = 3, n_segs: int = 2) -> Scene:
    """1024^2 grid over [0,4096)^2: 200 convex polygons with 4..8 vertices on a
    circle of radius uniform 20..120 (integer vertices, strict hull), circles
    >= 1 unit apart; 3 integer point sources + 2 segment sources (length
    uniform 50..400, uniform direction, integer endpoints), all clear of every
    polygon's bounding circle."""
    rng = SplitMix64(seed * 0x1000193 + 23)
    polys, circles = _place_convex_polys(rng, W, n_polys)
    pts = [_random_point_source(rng, W, circles) for _ in range(n_points)]
    segs = [_random_segment_source(rng, W, circles) for _ in range(n_segs)]
    return Scene((W, W), (N, N), polys, np.array(pts).reshape(-1, 2),
                 np.array(segs).reshape(-1, 4), name=f"plain_polys_{N}", seed=seed,
                 meta={"n_polys": len(polys)})


def maze(seed: int = 0, cells: int = 64, cell: int = 256, thick: int = 16,
         N: int = 4096, n_points: int = 4) -> Scene:
    """Randomised-DFS perfect maze of cells x cells, cell side 256 world units
    (world 16384^2 for 64 cells), grid N^2. Every remaining wall is a
    thick x (cell + thick) rectangle spanning post to post including both
    posts, so neighbouring walls overlap at posts; outer walls are centred on
    the world boundary. Sources: one exit segment 4 units inside the bottom
    outer wall's inner face (y = thick/2 + 4) across a seeded boundary cell
    (x from c*cell + 12 to c*cell + cell - 12), and n_points point sources at
    distinct seeded cell centres."""
    rng = SplitMix64(seed * 0x1000193 + 37)
    W = cells * cell
    ht = thick // 2
    # horizontal wall h[cx][cy] lies on y = cy*cell between x = cx*cell..(cx+1)*cell
    hwall = [[True] * (cells + 1) for _ in range(cells)]
    vwall = [[True] * cells for _ in range(cells + 1)]  # v[cx][cy]: x = cx*cell
    visited = [[False] * cells for _ in range(cells)]
    sx, sy = rng.randint(0, cells - 1), rng.randint(0, cells - 1)
    stack = [(sx, sy)]
    visited[sx][sy] = True
    while stack:
        x, y = stack[-1]
        nbrs = [(dx, dy) for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1))
                if 0 <= x + dx < cells and 0 <= y + dy < cells
                and not visited[x + dx][y + dy]]
        if not nbrs:
            stack.pop()
            continue
        dx, dy = nbrs[rng.randint(0, len(nbrs) - 1)]
        nx, ny = x + dx, y + dy
        if dx == 1:
            vwall[x + 1][y] = False
        elif dx == -1:
            vwall[x][y] = False
        elif dy == 1:
            hwall[x][y + 1] = False
        else:
            hwall[x][y] = False
        visited[nx][ny] = True
        stack.append((nx, ny))
    polys = []
    for cx in range(cells):
        for cy in range(cells + 1):
            if hwall[cx][cy]:
                x0, x1 = cx * cell - ht, (cx + 1) * cell + ht
                y0, y1 = cy * cell - ht, cy * cell + ht
                polys.append(np.array([(x0, y0), (x1, y0), (x1, y1), (x0, y1)], np.int32))
    for cx in range(cells + 1):
        for cy in range(cells):
            if vwall[cx][cy]:
                x0, x1 = cx * cell - ht, cx * cell + ht
                y0, y1 = cy * cell - ht, (cy + 1) * cell + ht
                polys.append(np.array([(x0, y0), (x1, y0), (x1, y1), (x0, y1)], np.int32))
    c = rng.randint(0, cells - 1)
    y_exit = float(ht + 4)
    segs = [(float(c * cell + 12), y_exit, float((c + 1) * cell - 12), y_exit)]
    chosen = set()
    pts = []
    while len(pts) < n_points:
        px, py = rng.randint(0, cells - 1), rng.randint(0, cells - 1)
        if (px, py) in chosen:
            continue
        chosen.add((px, py))
        pts.append((float(px * cell + cell // 2), float(py * cell + cell // 2)))
    return Scene((W, W), (N, N), polys, np.array(pts), np.array(segs),
                 name=f"maze_{cells}x{cells}_{N}", seed=seed,
                 meta={"cells": cells, "cell": cell, "thick": thick,
                       "n_walls": len(polys)})


def batched(seed: int = 0, n_scenes: int = 256, W: int = 4096,
            sides=(128, 256, 512, 1024), poly_range=(10, 500),
            src_range=(1, 6)) -> List[Scene]:
    """Independent scenes for one batched launch: grid side uniform in
    {128, 256, 512, 1024} over a 4096^2 world, 10..500 convex polygons as in
    the 1024^2 workload, 1..6 sources each a point or a segment (p = 1/2)."""
    rng = SplitMix64(seed * 0x1000193 + 51)
    out = []
    for s in range(n_scenes):
        sub = SplitMix64(rng.next_u64())
        N = sides[sub.randint(0, len(sides) - 1)]
        n_poly = sub.randint(*poly_range)
        n_src = sub.randint(*src_range)
        polys, circles = _place_convex_polys(sub, W, n_poly)
        pts, segs = [], []
        for _ in range(n_src):
            if sub.uniform() < 0.5:
                pts.append(_random_point_source(sub, W, circles))
            else:
                segs.append(_random_segment_source(sub, W, circles))
        out.append(Scene((W, W), (N, N), polys, np.array(pts).reshape(-1, 2),
                         np.array(segs).reshape(-1, 4), name=f"batched_{s}",
                         seed=seed, meta={"index": s, "n_polys": len(polys)}))
    return out


def differentiable(seed: int = 0, W: int = 8192, N: int = 2048, n_polys: int = 150,
                   n_points: int = 4, n_segs: int = 1, n_agents: int = 100_000) -> Scene:
    """2048^2 grid over [0,8192)^2 with 150 convex polygons, 4 movable FP32
    point sources and 1 movable FP32 segment source; 100k agents drawn
    uniformly with replacement among pixels whose centre lies outside every
    polygon's bounding circle (a conservative stand-in for free space)."""
    rng = SplitMix64(seed * 0x1000193 + 67)
    polys, circles = _place_convex_polys(rng, W, n_polys)
    pts = [_random_point_source(rng, W, circles, integer=False) for _ in range(n_points)]
    segs = [_random_segment_source(rng, W, circles, integer=False) for _ in range(n_segs)]
    h = W / N
    # conservative free-pixel mask from bounding circles (vectorised)
    ii = (np.arange(N) + 0.5) * h
    free = np.ones((N, N), dtype=bool)
    for (ox, oy, orb) in circles:
        r = orb + 1.0
        j0, j1 = max(0, int((oy - r) / h) - 1), min(N, int((oy + r) / h) + 2)
        i0, i1 = max(0, int((ox - r) / h) - 1), min(N, int((ox + r) / h) + 2)
        X = ii[i0:i1][None, :] - ox
        Y = ii[j0:j1][:, None] - oy
        free[j0:j1, i0:i1] &= (X * X + Y * Y) > r * r
    cand = np.flatnonzero(free.reshape(-1))
    picks = np.array([cand[rng.randint(0, len(cand) - 1)] for _ in range(n_agents)],
                     dtype=np.int64)
    agents = np.stack([picks % N, picks // N], axis=1).astype(np.int32)
    return Scene((W, W), (N, N), polys, np.array(pts), np.array(segs).reshape(-1, 4),
                 name=f"differentiable_{N}", seed=seed,
                 meta={"n_polys": len(polys)}, agents=agents)


def tiny(seed: int = 0, W: int = 48, N: int = 48, n_polys: int = 3, n_points: int = 1,
         n_segs: int = 0, r=(3.0, 9.0), k=(3, 6)) -> Scene:
    """Small scenes for brute-force cross-checks (few polygons, small grid)."""
    rng = SplitMix64(seed * 0x1000193 + 79)
    polys, circles = _place_convex_polys(rng, W, n_polys, r[0], r[1], k[0], k[1])
    pts = [_random_point_source(rng, W, circles) for _ in range(n_points)]
    segs = [_random_segment_source(rng, W, circles, len_lo=4.0, len_hi=W / 3.0)
            for _ in range(n_segs)]
    return Scene((W, W), (N, N), polys, np.array(pts).reshape(-1, 2),
                 np.array(segs).reshape(-1, 4), name=f"tiny_{seed}", seed=seed)


def empty_scene(W: int = 64, N: int = 64, points=(), segs=()) -> Scene:
    return Scene((W, W), (N, N), [], np.array(points, dtype=np.float64).reshape(-1, 2),
                 np.array(segs, dtype=np.float64).reshape(-1, 4), name="empty")


def single_square(W: int = 64, N: int = 64, square=(24, 24, 40, 40), source=(10.0, 30.0)) -> Scene:
    x0, y0, x1, y1 = square
    poly = np.array([(x0, y0), (x1, y0), (x1, y1), (x0, y1)], np.int32)
    return Scene((W, W), (N, N), [poly], np.array([source], dtype=np.float64),
                 np.zeros((0, 4)), name="single_square")


def profiling_map(k: int = 8, W: int = 1000, N: int = 1000, seed: int = 0) -> Scene:
    """k x k uniform rows of axis-aligned squares (P = k^2 polygons, V = 4P),
    each square half the row pitch wide and centred in its cell, with one
    seeded integer point source in a corridor between squares."""
    rng = SplitMix64(seed * 0x1000193 + 97)
    pitch = W // k
    side = pitch // 2
    polys, boxes = [], []
    for a in range(k):
        for b in range(k):
            x0 = a * pitch + (pitch - side) // 2
            y0 = b * pitch + (pitch - side) // 2
            polys.append(np.array([(x0, y0), (x0 + side, y0), (x0 + side, y0 + side),
                                   (x0, y0 + side)], np.int32))
            boxes.append((x0, y0, x0 + side, y0 + side))
    while True:
        x, y = rng.randint(1, W - 1), rng.randint(1, W - 1)
        if all(not (b[0] <= x <= b[2] and b[1] <= y <= b[3]) for b in boxes):
            break
    return Scene((W, W), (N, N), polys, np.array([(float(x), float(y))]),
                 np.zeros((0, 4)), name=f"profiling_{k * k}", seed=seed)


def profiling_sources(k: int = 8, n: int = 100, W: int = 1000, seed: int = 0) -> np.ndarray:
    """n seeded integer source positions for profiling_map(k, W): uniform in
    the world, kept when outside every (closed) square, so each is free."""
    rng = SplitMix64(seed * 0x1000193 + 131)
    pitch = W // k
    side = pitch // 2
    out = []
    while len(out) < n:
        x, y = rng.randint(1, W - 1), rng.randint(1, W - 1)
        a, b = x // pitch, y // pitch
        x0, y0 = a * pitch + (pitch - side) // 2, b * pitch + (pitch - side) // 2
        if a < k and b < k and x0 <= x <= x0 + side and y0 <= y <= y0 + side:
            continue
        out.append((float(x), float(y)))
    return np.array(out)


def maze_source_frames(scene: Scene, frames: int, seed: int = 0, step: int = 6):
    """Seeded per-frame sources for a maze() scene (maps of moving sources):
    frame 0 is the scene's own sources; after it every point source takes an
    integer random walk (each axis moves by a seeded step in [-step, step])
    clamped to its cell's free interior, 8 units clear of the walls, and the
    exit segment slides sideways by a clamped walk of at most 3 units (its
    ends stay 9 units clear of the side walls). Integer arithmetic only, so
    both machines draw the same frames. Returns float32 arrays points
    (frames, n_points, 2) and segs (frames, n_segs, 4)."""
    cell, thick = int(scene.meta["cell"]), int(scene.meta["thick"])
    ht = thick // 2
    rng = SplitMix64(seed * 0x1000193 + 977)
    p0 = np.asarray(scene.points, np.float64).reshape(-1, 2)
    s0 = np.asarray(scene.segs, np.float64).reshape(-1, 4)
    pts = np.zeros((frames, len(p0), 2), np.float32)
    segs = np.zeros((frames, len(s0), 4), np.float32)
    cur = [[int(x), int(y)] for x, y in p0]
    lo_hi = []
    for x, y in cur:
        cx, cy = x // cell, y // cell
        lo_hi.append((cx * cell + ht + 8, (cx + 1) * cell - ht - 8, cy * cell + ht + 8, (cy + 1) * cell - ht - 8))
    shift = 0
    for f in range(frames):
        if f > 0:
            for i, (x0, x1, y0, y1) in enumerate(lo_hi):
                cur[i][0] = min(x1, max(x0, cur[i][0] + rng.randint(-step, step)))
                cur[i][1] = min(y1, max(y0, cur[i][1] + rng.randint(-step, step)))
            shift = min(3, max(-3, shift + rng.randint(-1, 1)))
        for i in range(len(cur)):
            pts[f, i] = cur[i]
        for i in range(len(s0)):
            segs[f, i] = (s0[i, 0] + shift, s0[i, 1], s0[i, 2] + shift, s0[i, 3])
    return pts, segs


def maze_agents(scene: Scene, n: int, seed: int = 0) -> np.ndarray:
    """n seeded agent pixels (column, row) for a maze() scene: uniform in the
    free interior of uniformly drawn cells, 16 units clear of the wall centre
    lines, so every agent pixel is free and reached."""
    cells, cell, thick = (int(scene.meta[k]) for k in ("cells", "cell", "thick"))
    ht = thick // 2
    rng = SplitMix64(seed * 0x1000193 + 1301)
    W, N = scene.world[0], scene.grid[0]
    out = np.zeros((n, 2), np.int32)
    for k in range(n):
        cx, cy = rng.randint(0, cells - 1), rng.randint(0, cells - 1)
        x = rng.randint(cx * cell + ht + 16, (cx + 1) * cell - ht - 16)
        y = rng.randint(cy * cell + ht + 16, (cy + 1) * cell - ht - 16)
        out[k] = (x * N // W, y * N // W)
    return out
