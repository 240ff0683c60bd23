"""Seeded input generators: the per-frame moving sources of a maze stay
valid (the oracle, which checks sources with its own exact predicates,
accepts every frame), start at the scene's sources and are reproducible."""
import numpy as np

import scenegen as sg


def test_maze_source_frames_are_free_and_reproducible(oracle_mod):
    scene = sg.maze(2, cells=8, N=256)
    pts, segs = sg.maze_source_frames(scene, 12, seed=4)
    again = sg.maze_source_frames(scene, 12, seed=4)
    assert np.array_equal(pts, again[0]) and np.array_equal(segs, again[1])
    assert np.array_equal(pts[0], np.asarray(scene.points, np.float32))
    assert np.array_equal(segs[0], np.asarray(scene.segs, np.float32))
    assert np.abs(np.diff(pts, axis=0)).max() <= 6
    assert np.abs(segs[:, :, [0, 2]] - segs[:1, :, [0, 2]]).max() <= 3
    assert np.array_equal(segs[:, :, [1, 3]], np.broadcast_to(segs[:1, :, [1, 3]], segs[:, :, [1, 3]].shape))
    assert len(np.unique(pts.reshape(len(pts), -1), axis=0)) > 1
    for f in range(len(pts)):
        moved = sg.Scene(scene.world, scene.grid, scene.polys, pts[f].astype(np.float64),
                         segs[f].astype(np.float64))
        oracle_mod.Oracle(moved, nthreads=2)  # raises OracleError on a non-free source
