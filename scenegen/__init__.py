"""Seeded synthetic scene generators for shortest-path-map workloads.

This package only draws random scenes (obstacle polygons, point and segment
sources, agent samples) and serialises them. It holds none of the SPM
arithmetic: no visibility, distance or argmin code lives here. Both the CUDA
library's tests/benchmarks and the CPU oracle consume its output as plain data.
"""
from .scenes import (  # noqa: F401
    Scene,
    SplitMix64,
    plain_rects,
    plain_polys,
    maze,
    batched,
    differentiable,
    tiny,
    empty_scene,
    single_square,
    profiling_map,
    profiling_sources,
    maze_source_frames,
    maze_agents,
    load_scene,
    save_scene,
)
