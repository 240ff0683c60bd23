"""CPU FP64 oracle for shortest-path maps -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package. It shares no code with the CUDA
library (``paper_1805_08500_gb300``) and never imports it.

``spm_oracle.c`` holds the definition-level computation (Dijkstra over the
visibility graph, then a per-pixel exact min over visible generators);
``sequential.py`` restates the paper's Procedures 1-4 one generator at a time
for tiny scenes, as a second independent algorithm used to pin the first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "spm_oracle.c")
_lock = threading.Lock()
_lib = None

K_POINT, K_SEGA, K_SEGB, K_SEGI, K_VERT = range(5)
CONE_NONE, CONE_LEFT, CONE_RIGHT, CONE_EMPTY = range(4)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=gnu11", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int,
                                   f64p, ctypes.c_int, f64p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_char_p,
                                   ctypes.c_int]
        lib.orc_free.argtypes = [P]
        lib.orc_info.argtypes = [P, i32p]
        lib.orc_generators.argtypes = [P, i32p, i32p, i64p, f64p, f64p, i32p, i32p,
                                       i64p, i64p]
        lib.orc_pixels.argtypes = [P, ctypes.c_int, i32p, f64p, i32p, f64p, i32p,
                                   ctypes.c_int, ctypes.c_int]
        lib.orc_visible.restype = ctypes.c_int
        lib.orc_visible.argtypes = [P] + [ctypes.c_longlong] * 4
        lib.orc_keys.argtypes = [P, ctypes.c_int, i32p, i32p, f64p]
        lib.orc_keys.restype = None
        lib.orc_points.argtypes = [P, ctypes.c_int, i64p, f64p, i32p]
        lib.orc_points.restype = None
        lib.orc_root_link.restype = ctypes.c_int
        lib.orc_root_link.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      f64p, ctypes.POINTER(ctypes.c_double)]
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Oracle:
    """Scene + vertex costs computed on the CPU in FP64.

    ``use_cone=True`` restricts obstacle-vertex generators to their shadow cone
    behind their parent (the labelling the library must reproduce);
    ``use_cone=False`` is the unrestricted textbook minimum (same distances).
    ``snap="pixel"`` decides a source's visibility at its position rounded to
    the coarse lattice (scale ``Sp``, at most 15 bits over the scene) that the
    GPU library uses; ``snap="fine"`` at its position rounded to the oracle's
    own lattice (scale ``S``, 24 bits), within 1/(2S) of where it is. Lattice
    coordinates (``lxy``, ``pixel_lattice``, ``points``) are in units of 1/S.
    """

    def __init__(self, scene, nthreads: int | None = None, use_cone: bool = True, snap: str = "pixel"):
        lib = _load()
        self.scene = scene
        self.nthreads = nthreads or default_threads()
        self.use_cone = bool(use_cone)
        if snap not in ("pixel", "fine"):
            raise ValueError("snap is 'pixel' or 'fine'")
        self.snap = snap
        off, xy = scene.flat()
        pts = np.ascontiguousarray(scene.points, dtype=np.float64).reshape(-1)
        segs = np.ascontiguousarray(scene.segs, dtype=np.float64).reshape(-1)
        if pts.size == 0:
            pts = np.zeros(1, np.float64)
        if segs.size == 0:
            segs = np.zeros(1, np.float64)
        if xy.size == 0:
            xy = np.zeros(2, np.int32)
        st = ctypes.c_int(0)
        err = ctypes.create_string_buffer(256)
        self._h = lib.orc_create(scene.world[0], scene.world[1], scene.grid[0],
                                 scene.grid[1], len(scene.polys), off, xy,
                                 len(scene.points), pts, len(scene.segs), segs,
                                 self.nthreads, int(self.use_cone), int(snap == "fine"),
                                 ctypes.byref(st), err, 256)
        if not self._h:
            raise OracleError(f"oracle rejected scene (code {st.value}): "
                              f"{err.value.decode()}")
        info = np.zeros(6, np.int32)
        lib.orc_info(self._h, info)
        self.n_gen, self.n_src, self.n_vert, self.S, self.n_poly, self.Sp = (int(v) for v in info)
        n = self.n_gen
        self.kind = np.zeros(n, np.int32)
        self.sidx = np.zeros(n, np.int32)
        self.lxy = np.zeros(2 * n, np.int64)
        self.txy = np.zeros(2 * n, np.float64)
        self.cost = np.zeros(n, np.float64)
        self.parent = np.zeros(n, np.int32)
        self.cside = np.zeros(n, np.int32)
        self.cdir = np.zeros(2 * n, np.int64)
        self.wedge = np.zeros(4 * n, np.int64)
        if n:
            lib.orc_generators(self._h, self.kind, self.sidx, self.lxy, self.txy,
                               self.cost, self.parent, self.cside, self.cdir, self.wedge)
        self.lxy = self.lxy.reshape(-1, 2)
        self.txy = self.txy.reshape(-1, 2)
        self.cdir = self.cdir.reshape(-1, 2)
        self.wedge = self.wedge.reshape(-1, 4)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    # ------------------------------------------------------------------
    def pixels(self, ij):
        """Field at pixels ij (n,2) = (column, row). Returns
        (dist, parent, second_dist, second_parent)."""
        ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
        n = ij.shape[0]
        dist = np.zeros(n, np.float64)
        par = np.zeros(n, np.int32)
        d2 = np.zeros(n, np.float64)
        p2 = np.zeros(n, np.int32)
        if n:
            _lib.orc_pixels(self._h, n, ij.reshape(-1), dist, par, d2, p2,
                            self.nthreads, int(self.use_cone))
        return dist, par, d2, p2

    def field(self):
        """Full field as (Ny, Nx) arrays (dist, parent, second, second_parent)."""
        Nx, Ny = self.scene.grid
        jj, ii = np.meshgrid(np.arange(Ny, dtype=np.int32), np.arange(Nx, dtype=np.int32),
                             indexing="ij")
        ij = np.stack([ii.reshape(-1), jj.reshape(-1)], axis=1)
        d, p, d2, p2 = self.pixels(ij)
        return (d.reshape(Ny, Nx), p.reshape(Ny, Nx), d2.reshape(Ny, Nx),
                p2.reshape(Ny, Nx))

    def keys(self, ij, gens):
        """Key of generator gens[n] at pixel ij[n] (inf when that generator is
        not valid there): to check a tied alternative parent."""
        ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
        gens = np.ascontiguousarray(np.asarray(gens, dtype=np.int32).reshape(-1))
        out = np.empty(len(gens), np.float64)
        if len(gens):
            _lib.orc_keys(self._h, len(gens), ij.reshape(-1), gens, out)
        return out

    def points(self, lxy):
        """Field (dist, parent) at arbitrary lattice points lxy (n, 2), world
        coordinates lxy / S (Sec. 6: exact point queries)."""
        lxy = np.ascontiguousarray(np.asarray(lxy, dtype=np.int64).reshape(-1, 2))
        n = lxy.shape[0]
        dist = np.zeros(n, np.float64)
        par = np.zeros(n, np.int32)
        if n:
            _lib.orc_points(self._h, n, lxy.reshape(-1), dist, par)
        return dist, par

    def visible(self, a, b) -> bool:
        """Exact visibility between two lattice points."""
        return bool(_lib.orc_visible(self._h, int(a[0]), int(a[1]), int(b[0]), int(b[1])))

    def pixel_lattice(self, i, j):
        Wx, Wy = (int(v) for v in self.scene.world)
        Nx, Ny = (int(v) for v in self.scene.grid)
        i, j = int(i), int(j)
        return ((2 * i + 1) * self.S * Wx // (2 * Nx), (2 * j + 1) * self.S * Wy // (2 * Ny))

    def root_link(self, i, j, first_parent):
        """(root generator, last point before it (true xy), foot parameter t)."""
        x = np.zeros(2, np.float64)
        t = ctypes.c_double(0.0)
        g = _lib.orc_root_link(self._h, int(i), int(j), int(first_parent), x,
                               ctypes.byref(t))
        return g, x, t.value

    # ------------------------------------------------------------------
    def agent_loss_and_grad(self, agents):
        """loss = mean oracle distance over agents (pixel indices, (n,2));
        gradient w.r.t. point sources (n_p,2) and segment endpoints (n_s,4)
        from the root link of each agent's parent chain: a point root s with
        last point x gives (s - x)/|s - x|; a segment interior with unit normal
        n toward x and foot parameter t gives -(1 - t) n and -t n on A and B."""
        agents = np.asarray(agents, dtype=np.int32).reshape(-1, 2)
        uniq, inv = np.unique(agents, axis=0, return_inverse=True)
        d, p, _, _ = self.pixels(uniq)
        if not np.all(np.isfinite(d)):
            raise OracleError("an agent sits on an unreached or non-free pixel")
        loss = float(np.mean(d[inv.reshape(-1)]))
        counts = np.bincount(inv.reshape(-1), minlength=len(uniq)).astype(np.float64)
        n_p, n_s = len(self.scene.points), len(self.scene.segs)
        gp = np.zeros((n_p, 2))
        gs = np.zeros((n_s, 4))
        for k in range(len(uniq)):
            g, x, t = self.root_link(uniq[k, 0], uniq[k, 1], p[k])
            w = counts[k] / len(agents)
            kind = self.kind[g]
            if kind == K_SEGI:
                s = self.sidx[g]
                A = self.scene.segs[s, :2]
                B = self.scene.segs[s, 2:]
                u = B - A
                f = A + t * u
                nv = x - f
                nn = np.hypot(*nv)
                if nn > 0:
                    nv = nv / nn
                    gs[s, :2] += w * (-(1.0 - t) * nv)
                    gs[s, 2:] += w * (-t * nv)
            else:
                sxy = self.txy[g]
                dv = sxy - x
                nn = np.hypot(*dv)
                if nn > 0:
                    dv = dv / nn
                    if kind == K_POINT:
                        gp[self.sidx[g]] += w * dv
                    elif kind == K_SEGA:
                        gs[self.sidx[g], :2] += w * dv
                    elif kind == K_SEGB:
                        gs[self.sidx[g], 2:] += w * dv
        return loss, gp, gs
