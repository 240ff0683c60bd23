"""GB300 shortest-path maps (arxiv 1805.08500) -- Python binding.

A thin ctypes layer over ``libspm_gb300.so`` (the C ABI of ``include/spm.h``):
functions carry the C names and only marshal arguments (tensors/arrays to
pointers, status codes to exceptions). Every step of the computation runs in
the library's CUDA kernels; there is no CPU fallback. PyTorch supplies device
memory and streams only.

The library must have been built in-tree (``__graft_entry__.build()`` or
``python paper_1805_08500_gb300/build.py``); importing the compute entry
points without it raises ``SpmLibraryMissing``.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the product library; SPM_GB300_LIB may name an instrumentation build of it
# (build.py --counters / --clocks) for a profiling session
LIB_PATH = os.environ.get("SPM_GB300_LIB") or os.path.join(_HERE, "libspm_gb300.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "spm.h")

SPM_OK = 0
STATUS_NAMES = {0: "SPM_OK", 1: "SPM_ERR_INVALID_ARG", 2: "SPM_ERR_BAD_GEOMETRY",
                3: "SPM_ERR_OOM", 4: "SPM_ERR_CUDA", 5: "SPM_ERR_NOT_CONVERGED",
                6: "SPM_ERR_TIMEOUT", 7: "SPM_ERR_CAPACITY"}
(SPM_ERR_INVALID_ARG, SPM_ERR_BAD_GEOMETRY, SPM_ERR_OOM, SPM_ERR_CUDA, SPM_ERR_NOT_CONVERGED,
 SPM_ERR_TIMEOUT, SPM_ERR_CAPACITY) = range(1, 8)
KIND_POINT, KIND_SEG_A, KIND_SEG_B, KIND_SEG_INTERIOR, KIND_VERTEX = range(5)


class SpmLibraryMissing(RuntimeError):
    pass


class SpmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}"
                         + (f" ({msg})" if msg else ""))


class SpmTuning(ctypes.Structure):
    _fields_ = [("flood_mode", ctypes.c_int32), ("hidden_chunk", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("maps", ctypes.c_int32), ("fixpoint_start", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class _Desc(ctypes.Structure):
    _fields_ = [("world_w", ctypes.c_int32), ("world_h", ctypes.c_int32),
                ("grid_w", ctypes.c_int32), ("grid_h", ctypes.c_int32),
                ("n_polys", ctypes.c_int32), ("poly_offsets", ctypes.c_void_p),
                ("poly_xy", ctypes.c_void_p), ("n_points", ctypes.c_int32),
                ("point_xy", ctypes.c_void_p), ("n_segments", ctypes.c_int32),
                ("seg_xyxy", ctypes.c_void_p)]


_lib = None


def declared_symbols() -> list:
    """Entry points declared in include/spm.h."""
    with open(HEADER_PATH) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(spm_\w+)\s*\(", text, re.M)))


def load_library():
    """Load libspm_gb300.so (raises SpmLibraryMissing when it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise SpmLibraryMissing(
            f"{LIB_PATH} is missing: build it with __graft_entry__.build(); "
            "there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    sigs = {
        "spm_scene_create": ([ctypes.POINTER(_Desc), ctypes.POINTER(P)], I32),
        "spm_scene_destroy": ([P], None),
        "spm_scene_update_sources": ([P, P, P], I32),
        "spm_scene_update_sources_device": ([P, P, P, P], I32),
        "spm_compute": ([P, P, P, P], I32),
        "spm_compute_rows": ([P, P, I32, I32, P, P], I32),
        "spm_compute_sequential": ([P, P, P, P], I32),
        "spm_compute_host": ([P, P, P, P], I32),
        "spm_compute_batched": ([P, I32, P, P, P], I32),
        "spm_batch_create": ([P, I32, P, P, P], I32),
        "spm_batch_compute": ([P, P], I32),
        "spm_batch_destroy": ([P], None),
        "spm_batch_phase_ms": ([P, P, P], I32),
        "spm_scene_sync": ([P, P], I32),
        "spm_query_parent": ([P, F, F, P, P], I32),
        "spm_query_exact": ([P, F, F, P, P], I32),
        "spm_extract_path": ([P, F, F, P, I32, P], I32),
        "spm_scene_generators": ([P, P, P, P, P], I32),
        "spm_scene_info": ([P, P], I32),
        "spm_agents_forward": ([P, P, P, I32, P, P, P, P], I32),
        "spm_agents_tape_bytes": ([I32], I64),
        "spm_agents_backward": ([P, P, P, I32, P, P], I32),
        "spm_scene_phase_ms": ([P, P, P, P], I32),
        "spm_agents_backward_noalloc": ([P, P, P, I32, P, P, P], I32),
        "spm_scene_get_tuning": ([P, P], I32),
        "spm_scene_set_tuning": ([P, P], I32),
        "spm_scene_autotune": ([P, P, P], I32),
        "spm_status_string": ([I32], ctypes.c_char_p),
        "spm_last_error": ([P], ctypes.c_char_p),
        "spm_debug_fail_alloc_after": ([I32], None),
        "spm_debug_set_round_cap": ([I32], None),
        "spm_debug_set_many_cta_fixpoint": ([I32], None),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str, handle=None):
    if st != SPM_OK:
        msg = load_library().spm_last_error(handle)
        raise SpmError(st, where, msg.decode() if msg else "")


def _ptr(x):
    """Raw address of a torch tensor, numpy array or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover - torch missing
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C entry points, same names
# ---------------------------------------------------------------------------

def spm_scene_create(scene):
    """Create a library scene from a ``scenegen.Scene``-like object (world,
    grid, polys, points, segs). Returns an opaque handle (int)."""
    lib = load_library()
    off, xy = _flat_polys(scene.polys)
    pts = np.ascontiguousarray(np.asarray(scene.points, np.float32).reshape(-1))
    segs = np.ascontiguousarray(np.asarray(scene.segs, np.float32).reshape(-1))
    d = _Desc(int(scene.world[0]), int(scene.world[1]), int(scene.grid[0]), int(scene.grid[1]),
              len(scene.polys), off.ctypes.data if len(off) else None,
              xy.ctypes.data if len(xy) else None, pts.size // 2,
              pts.ctypes.data if pts.size else None, segs.size // 4,
              segs.ctypes.data if segs.size else None)
    h = ctypes.c_void_p()
    _check(lib.spm_scene_create(ctypes.byref(d), ctypes.byref(h)), "spm_scene_create")
    return h.value


def spm_scene_destroy(handle):
    if handle:
        load_library().spm_scene_destroy(handle)


def spm_scene_update_sources(handle, points, segs):
    pts = np.ascontiguousarray(np.asarray(points, np.float32).reshape(-1))
    sg = np.ascontiguousarray(np.asarray(segs, np.float32).reshape(-1))
    _check(load_library().spm_scene_update_sources(
        handle, pts.ctypes.data if pts.size else None, sg.ctypes.data if sg.size else None),
        "spm_scene_update_sources", handle)


def spm_scene_update_sources_device(handle, stream, points_dev, segs_dev):
    """Move the sources from device buffers (float32, contiguous, on the
    scene's device; None when the count is 0), stream-ordered."""
    for t in (points_dev, segs_dev):
        if t is not None and hasattr(t, "is_cuda"):
            if not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous() or not t.is_floating_point():
                raise ValueError("device sources must be contiguous float32 CUDA tensors")
    pp = _ptr(points_dev) if points_dev is not None and _numel(points_dev) else None
    sp = _ptr(segs_dev) if segs_dev is not None and _numel(segs_dev) else None
    _check(load_library().spm_scene_update_sources_device(handle, _stream_handle(stream), pp, sp),
           "spm_scene_update_sources_device", handle)


def _numel(x):
    return x.numel() if hasattr(x, "numel") else int(np.size(x))


def spm_compute(handle, stream, dist, parent):
    _check(load_library().spm_compute(handle, _stream_handle(stream), _ptr(dist), _ptr(parent)),
           "spm_compute", handle)


def spm_compute_sequential(handle, stream, dist, parent):
    _check(load_library().spm_compute_sequential(handle, _stream_handle(stream), _ptr(dist), _ptr(parent)),
           "spm_compute_sequential", handle)


def spm_compute_rows(handle, stream, row0, row1, dist, parent):
    _check(load_library().spm_compute_rows(handle, _stream_handle(stream), int(row0), int(row1), _ptr(dist),
                                           _ptr(parent)), "spm_compute_rows", handle)


def row_slabs(grid_h: int, tile: int, world: int):
    """Tile-aligned row slabs [row0, row1) of a grid, one per rank: whole
    tile rows dealt as evenly as possible, the last slab ending at grid_h."""
    tiles = (grid_h + tile - 1) // tile
    out = []
    for r in range(world):
        t0, t1 = tiles * r // world, tiles * (r + 1) // world
        out.append((min(t0 * tile, grid_h), min(t1 * tile, grid_h)))
    return out


def spm_compute_host(handle, stream, dist_host, parent_host):
    _check(load_library().spm_compute_host(handle, _stream_handle(stream), _ptr(dist_host),
                                           _ptr(parent_host)), "spm_compute_host", handle)


def spm_compute_batched(handles, stream, dists, parents):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*handles)
    D = (ctypes.c_void_p * n)(*[_ptr(d) for d in dists])
    Pp = (ctypes.c_void_p * n)(*[_ptr(p) for p in parents])
    _check(load_library().spm_compute_batched(H, n, _stream_handle(stream), D, Pp),
           "spm_compute_batched")


def spm_batch_create(handles, dists, parents):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*handles)
    D = (ctypes.c_void_p * n)(*[_ptr(d) for d in dists])
    Pp = (ctypes.c_void_p * n)(*[_ptr(p) for p in parents])
    out = ctypes.c_void_p()
    _check(load_library().spm_batch_create(H, n, D, Pp, ctypes.byref(out)), "spm_batch_create")
    return out.value


def spm_batch_compute(batch, stream=None):
    _check(load_library().spm_batch_compute(batch, _stream_handle(stream)), "spm_batch_compute")


def spm_batch_phase_ms(batch):
    """(vertex_ms, pixel_ms) of the last batch compute, from events inside its launch sequence."""
    v = ctypes.c_float()
    p = ctypes.c_float()
    _check(load_library().spm_batch_phase_ms(batch, ctypes.byref(v), ctypes.byref(p)), "spm_batch_phase_ms")
    return v.value, p.value


def spm_batch_destroy(batch):
    if batch:
        load_library().spm_batch_destroy(batch)


class Batch:
    """Scenes computed together; outputs are torch tensors, one pair per scene."""

    def __init__(self, scenes):
        self.scenes = list(scenes)
        self.outputs = [s.empty_outputs() for s in self.scenes]
        self.handle = spm_batch_create([s.handle for s in self.scenes],
                                       [o[0] for o in self.outputs], [o[1] for o in self.outputs])

    def compute(self, stream=None):
        spm_batch_compute(self.handle, stream)
        return self.outputs

    def phase_ms(self):
        return spm_batch_phase_ms(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            spm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spm_scene_sync(handle, stream=None):
    _check(load_library().spm_scene_sync(handle, _stream_handle(stream)), "spm_scene_sync", handle)


def spm_query_parent(handle, x, y):
    p = ctypes.c_int32()
    d = ctypes.c_float()
    _check(load_library().spm_query_parent(handle, float(x), float(y), ctypes.byref(p),
                                           ctypes.byref(d)), "spm_query_parent", handle)
    return p.value, d.value


def spm_query_exact(handle, x, y):
    """(parent, distance) at (x, y) itself, from the neighbouring pixels' parents."""
    p = ctypes.c_int32()
    d = ctypes.c_float()
    _check(load_library().spm_query_exact(handle, float(x), float(y), ctypes.byref(p),
                                          ctypes.byref(d)), "spm_query_exact", handle)
    return p.value, d.value


def spm_extract_path(handle, x, y, cap=4096):
    out = np.zeros(2 * cap, np.float32)
    n = ctypes.c_int32()
    _check(load_library().spm_extract_path(handle, float(x), float(y), out.ctypes.data, cap,
                                           ctypes.byref(n)), "spm_extract_path", handle)
    return out[:2 * n.value].reshape(-1, 2)


def spm_scene_get_tuning(handle):
    t = SpmTuning()
    _check(load_library().spm_scene_get_tuning(handle, ctypes.byref(t)), "spm_scene_get_tuning", handle)
    return {"flood_mode": t.flood_mode, "hidden_chunk": t.hidden_chunk, "tile": t.tile, "maps": t.maps,
            "fixpoint_start": t.fixpoint_start}


def spm_scene_set_tuning(handle, flood_mode, hidden_chunk, tile=0, maps=0, fixpoint_start=0):
    """fixpoint_start: 0 automatic, 1 from the sources, 2 from the tree of the
    scene's obstacle-vertex geodesic table (when it has one)."""
    t = SpmTuning(int(flood_mode), int(hidden_chunk), int(tile), int(maps), int(fixpoint_start))
    _check(load_library().spm_scene_set_tuning(handle, ctypes.byref(t)), "spm_scene_set_tuning", handle)


def spm_scene_autotune(handle, stream=None):
    t = SpmTuning()
    _check(load_library().spm_scene_autotune(handle, _stream_handle(stream), ctypes.byref(t)),
           "spm_scene_autotune", handle)
    return {"flood_mode": t.flood_mode, "hidden_chunk": t.hidden_chunk, "tile": t.tile, "maps": t.maps}


def spm_scene_info(handle):
    info = np.zeros(11, np.int64)
    _check(load_library().spm_scene_info(handle, info.ctypes.data), "spm_scene_info", handle)
    keys = ["n_gen", "n_src", "n_vert", "lattice_scale", "n_polys", "rounds", "edges", "tile",
            "flooded", "flood_mode", "kernels_per_compute"]
    return dict(zip(keys, (int(v) for v in info)))


def spm_scene_generators(handle):
    n = spm_scene_info(handle)["n_gen"]
    kind = np.zeros(n, np.int32)
    lat = np.zeros(2 * n, np.int32)
    cost = np.zeros(n, np.float64)
    par = np.zeros(n, np.int32)
    _check(load_library().spm_scene_generators(handle, kind.ctypes.data, lat.ctypes.data,
                                               cost.ctypes.data, par.ctypes.data),
           "spm_scene_generators", handle)
    return kind, lat.reshape(-1, 2), cost, par


def spm_agents_forward(handle, stream, agents, dist, parent, loss, tape=None):
    """Mean agent distance into loss; with tape (device buffer of
    spm_agents_tape_bytes(n) bytes) also records the backward's inputs."""
    n = int(agents.shape[0]) if hasattr(agents, "shape") else len(agents) // 2
    _check(load_library().spm_agents_forward(handle, _stream_handle(stream), _ptr(agents), n,
                                             _ptr(dist), _ptr(parent), _ptr(loss), _ptr(tape)),
           "spm_agents_forward", handle)


def spm_agents_tape_bytes(n: int) -> int:
    return int(load_library().spm_agents_tape_bytes(int(n)))


def empty_tape(n: int, device):
    """A device tape for n agents (16-byte aligned)."""
    import torch
    return torch.empty(max(spm_agents_tape_bytes(n), 16), dtype=torch.uint8, device=device)


def spm_agents_backward(handle, stream, tape, n, grad_points, grad_segs):
    _check(load_library().spm_agents_backward(handle, _stream_handle(stream), _ptr(tape), int(n),
                                              _ptr(grad_points), _ptr(grad_segs)), "spm_agents_backward", handle)


def spm_agents_backward_noalloc(handle, stream, agents, parent, grad_points, grad_segs):
    """Same gradient as spm_agents_forward + spm_agents_backward, but the
    library allocates nothing: its scratch is a fixed in-library array (see
    include/spm.h for the limits and the shared-scratch caveat)."""
    n = int(agents.shape[0]) if hasattr(agents, "shape") else len(agents) // 2
    _check(load_library().spm_agents_backward_noalloc(
        handle, _stream_handle(stream), _ptr(agents), n, _ptr(parent), _ptr(grad_points),
        _ptr(grad_segs)), "spm_agents_backward_noalloc", handle)


def spm_scene_phase_ms(handle):
    """(vertex_ms, cull_ms, pixel_ms) of the last compute, from the library's events."""
    v = ctypes.c_float()
    c = ctypes.c_float()
    p = ctypes.c_float()
    _check(load_library().spm_scene_phase_ms(handle, ctypes.byref(v), ctypes.byref(c), ctypes.byref(p)),
           "spm_scene_phase_ms", handle)
    return v.value, c.value, p.value


def spm_status_string(status: int) -> str:
    return load_library().spm_status_string(int(status)).decode()


def _flat_polys(polys):
    off = np.zeros(len(polys) + 1, np.int32)
    for i, p in enumerate(polys):
        off[i + 1] = off[i] + len(p)
    xy = (np.concatenate([np.asarray(p, np.int32).reshape(-1) for p in polys])
          if polys else np.zeros(0, np.int32)).astype(np.int32)
    return np.ascontiguousarray(off), np.ascontiguousarray(xy)


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Scene:
    """Owns one library scene; outputs are torch tensors on the scene's device."""

    def __init__(self, scene):
        import torch
        self.desc = scene
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle = spm_scene_create(scene)
        self.grid = (int(scene.grid[0]), int(scene.grid[1]))

    def close(self):
        if getattr(self, "handle", None):
            spm_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_outputs(self):
        import torch
        Nx, Ny = self.grid
        return (torch.empty((Ny, Nx), dtype=torch.float32, device=self.device),
                torch.empty((Ny, Nx), dtype=torch.int32, device=self.device))

    def compute_rows(self, row0, row1, dist, parent, stream=None):
        """Rows [row0, row1) of the map into the full-grid buffers (tile-aligned)."""
        spm_compute_rows(self.handle, stream, row0, row1, dist, parent)
        return dist, parent

    def compute(self, dist=None, parent=None, stream=None):
        if dist is None or parent is None:
            dist, parent = self.empty_outputs()
        spm_compute(self.handle, stream, dist, parent)
        return dist, parent

    def compute_sequential(self, dist=None, parent=None, stream=None):
        """The map by the paper's generator-sequential schedule (A/B baseline)."""
        if dist is None or parent is None:
            dist, parent = self.empty_outputs()
        spm_compute_sequential(self.handle, stream, dist, parent)
        return dist, parent

    def sync(self, stream=None):
        spm_scene_sync(self.handle, stream)

    def info(self):
        return spm_scene_info(self.handle)

    def generators(self):
        return spm_scene_generators(self.handle)

    def update_sources(self, points, segs):
        spm_scene_update_sources(self.handle, points, segs)

    def update_sources_device(self, points, segs, stream=None):
        """Move the sources from float32 CUDA tensors (n_points, 2) and
        (n_segs, 4), stream-ordered; a rejected move surfaces at sync()."""
        spm_scene_update_sources_device(self.handle, stream, points, segs)

    def autotune(self, stream=None, cache_key=None):
        """Pick the culling configuration: from the tuning cache when cache_key
        (a workload-class string) has an entry for this GPU, else by timing
        (spm_scene_autotune) and recording the result in the cache."""
        return autotune_cached(self, stream, cache_key)

    def tuning(self):
        return spm_scene_get_tuning(self.handle)

    def phase_ms(self):
        return spm_scene_phase_ms(self.handle)

    def query_parent(self, x, y):
        return spm_query_parent(self.handle, x, y)

    def query_exact(self, x, y):
        return spm_query_exact(self.handle, x, y)

    def extract_path(self, x, y, cap=4096):
        return spm_extract_path(self.handle, x, y, cap)


TUNING_CACHE = os.path.join(_HERE, "tuning_cache.json")


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def autotune_cached(scene: "Scene", stream=None, cache_key=None, path=TUNING_CACHE):
    import json
    cache = {}
    if os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    key = f"{cache_key}|{_gpu_name()}" if cache_key else None
    if key and key in cache:
        t = cache[key]
        spm_scene_set_tuning(scene.handle, t["flood_mode"], t["hidden_chunk"], t.get("tile", 0), t.get("maps", 0))
        return dict(t, source="cache")
    t = spm_scene_autotune(scene.handle, stream)
    if key:
        cache[key] = t
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return dict(t, source="measured")


def agent_loss(scene: "Scene", points, segs, agents):
    """Differentiable mean geodesic distance of agents (pixel indices, int32
    (n, 2) device tensor) w.r.t. the point sources (n_p, 2) and segment
    endpoints (n_s, 4): forward and backward run in the library's kernels.
    The sources move on the device (no host round trip); a move the library
    rejects keeps the previous sources and is reported by scene.sync()."""
    return _AgentLoss.apply(points, segs, scene, agents)


def _make_autograd():
    import torch

    class AgentLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, points, segs, scene, agents):
            # the sources move on the device: no host round trip in the step
            pts = points.detach().to(scene.device, torch.float32).contiguous()
            sgs = segs.detach().to(scene.device, torch.float32).contiguous()
            spm_scene_update_sources_device(scene.handle, None, pts.reshape(-1) if pts.numel() else None,
                                            sgs.reshape(-1) if sgs.numel() else None)
            dist, parent = scene.compute()
            loss = torch.empty((), dtype=torch.float32, device=scene.device)
            n = int(agents.shape[0])
            tape = empty_tape(n, scene.device)  # what the backward needs, from this forward
            spm_agents_forward(scene.handle, None, agents, dist, parent, loss, tape)
            ctx.scene = scene
            ctx.tape, ctx.n = tape, n
            ctx.shapes = (points.shape, segs.shape)
            ctx.devices = (points.device, segs.device)
            return loss

        @staticmethod
        def backward(ctx, grad_out):
            scene = ctx.scene
            gp = torch.zeros(ctx.shapes[0], dtype=torch.float32, device=scene.device)
            gs = torch.zeros(ctx.shapes[1], dtype=torch.float32, device=scene.device)
            spm_agents_backward(scene.handle, None, ctx.tape, ctx.n, gp if gp.numel() else None,
                                gs if gs.numel() else None)
            g = grad_out.to(scene.device)
            return (gp * g).to(ctx.devices[0]), (gs * g).to(ctx.devices[1]), None, None

    return AgentLoss


class _Lazy:
    _fn = None

    def apply(self, *args):
        if _Lazy._fn is None:
            _Lazy._fn = _make_autograd()
        return _Lazy._fn.apply(*args)


_AgentLoss = _Lazy()


def debug_read(kind: str):
    """Read and clear an instrumentation build's device counters: kind
    "pixels", "flood" or "vertex" (32 work counters each, SPM_COUNT build) or
    "pixel_clocks" / "flood_clocks" (8 phase clocks, SPM_TIME build). Raises
    AttributeError on the product library, which has none."""
    names = {"pixels": ("spm_debug_counters", 32), "flood": ("spm_debug_counters_flood", 32),
             "vertex": ("spm_debug_counters_vertex", 32), "pixel_clocks": ("spm_debug_times", 8),
             "flood_clocks": ("spm_debug_times_flood", 8)}
    name, n = names[kind]
    fn = getattr(load_library(), name)
    buf = (ctypes.c_ulonglong * n)()
    fn.argtypes = [ctypes.c_void_p]
    fn.restype = ctypes.c_int
    if fn(ctypes.addressof(buf)) != 0:
        raise SpmError(SPM_ERR_CUDA, name)
    return list(buf)

