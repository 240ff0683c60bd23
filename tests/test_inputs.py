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


def test_scene_files_round_trip_and_generators_are_seeded(tmp_path, oracle_mod):
    """A scene written to a file and read back is the same scene (so a
    failing case can be replayed); the generators are functions of their
    seed; and the oracle gives the same field for the reloaded scene."""
    for scene in (sg.plain_rects(3), sg.plain_polys(1, W=1024, N=64, n_polys=12, n_segs=1),
                  sg.maze(1, cells=4, N=64), sg.differentiable(2, W=512, N=64, n_polys=6, n_agents=50)):
        path = str(tmp_path / "scene.json")
        sg.save_scene(scene, path)
        back = sg.load_scene(path)
        assert back.world == tuple(scene.world) and back.grid == tuple(scene.grid)
        assert len(back.polys) == len(scene.polys)
        assert all(np.array_equal(a, b) for a, b in zip(back.polys, scene.polys))
        assert np.array_equal(back.points, np.asarray(scene.points, np.float64).reshape(-1, 2))
        assert np.array_equal(back.segs, np.asarray(scene.segs, np.float64).reshape(-1, 4))
        if scene.agents is not None:
            assert np.array_equal(back.agents, scene.agents)
    a, b = sg.plain_polys(5, W=1024, N=64, n_polys=12), sg.plain_polys(5, W=1024, N=64, n_polys=12)
    assert all(np.array_equal(p, q) for p, q in zip(a.polys, b.polys)) and np.array_equal(a.points, b.points)
    c = sg.plain_polys(6, W=1024, N=64, n_polys=12)
    assert not all(np.array_equal(p, q) for p, q in zip(a.polys, c.polys))
    s = sg.plain_rects(3)
    sg.save_scene(s, str(tmp_path / "r.json"))
    d1 = oracle_mod.Oracle(s, nthreads=2).field()[0]
    d2 = oracle_mod.Oracle(sg.load_scene(str(tmp_path / "r.json")), nthreads=2).field()[0]
    assert np.array_equal(d1, d2)
