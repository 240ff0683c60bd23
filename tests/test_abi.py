"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point include/spm.h declares; host-side validation rejects bad scenes
before touching CUDA; with no device the compute path fails loudly."""
import os
import subprocess

import numpy as np
import pytest

import scenegen as sg

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spm():
    import paper_1805_08500_gb300 as m
    from paper_1805_08500_gb300 import build
    build.build()
    m.load_library()
    return m


def test_exports_every_declared_symbol(spm):
    names = spm.declared_symbols()
    assert len(names) >= 15
    lib = spm.load_library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", spm.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported


def test_status_strings(spm):
    for code in range(8):
        assert spm.spm_status_string(code)


def _bad(spm, scene, code=2):
    with pytest.raises(spm.SpmError) as ei:
        spm.spm_scene_create(scene)
    assert ei.value.status == code, str(ei.value)


def test_rejects_bad_geometry_on_host(spm):
    sq = np.array([(10, 10), (20, 10), (20, 20), (10, 20)])
    Z = np.zeros((0, 4))
    _bad(spm, sg.Scene((32, 32), (32, 32), [sq], [(15.0, 15.0)], Z))          # source inside
    _bad(spm, sg.Scene((32, 32), (32, 32), [sq], [(10.0, 12.0)], Z))          # on the boundary
    _bad(spm, sg.Scene((32, 32), (32, 32), [sq], [(40.0, 12.0)], Z))          # outside the world
    _bad(spm, sg.Scene((32, 32), (32, 32), [sq], [(2.0, 2.0)], [(5.0, 15, 25, 15)]))  # crossing
    _bad(spm, sg.Scene((32, 32), (32, 32), [sq], [(2.0, 2.0)], [(5.0, 5, 5, 5)]))     # zero length
    nonconvex = np.array([(0, 0), (10, 0), (5, 2), (10, 10), (0, 10)])
    _bad(spm, sg.Scene((32, 32), (32, 32), [nonconvex], [(20.0, 20.0)], Z))
    collinear = np.array([(0, 0), (5, 0), (10, 0), (10, 10), (0, 10)])
    _bad(spm, sg.Scene((32, 32), (32, 32), [collinear], [(20.0, 20.0)], Z))
    big = np.array([(int(16 + 10 * np.cos(a)), int(16 + 10 * np.sin(a)))
                    for a in np.linspace(0, 2 * np.pi, 40, endpoint=False)])
    _bad(spm, sg.Scene((64, 64), (64, 64), [np.unique(big, axis=0)[:17]], [(60.0, 60.0)], Z))
    touch = [np.array([(0, 0), (4, 0), (4, 4), (0, 4)]), np.array([(4, 4), (8, 4), (8, 8), (4, 8)])]
    _bad(spm, sg.Scene((16, 16), (16, 16), touch, [(12.0, 2.0)], Z))           # single-point touch
    _bad(spm, sg.Scene((40000, 40000), (40000, 40000), [], [(3.0, 3.0)], Z))  # beyond lattice
    _bad(spm, sg.Scene((32, 32), (32, 32), [], np.zeros((0, 2)), Z), code=1)   # no source


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")
def test_no_device_fails_loudly(spm):
    s = sg.plain_rects(0)
    with pytest.raises(spm.SpmError) as ei:
        spm.spm_scene_create(s)
    assert ei.value.status == 4  # SPM_ERR_CUDA: no device, no CPU fallback


def test_missing_library_is_loud(tmp_path, monkeypatch):
    import paper_1805_08500_gb300 as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "LIB_PATH", os.path.join(str(tmp_path), "nope.so"))
    with pytest.raises(m.SpmLibraryMissing):
        m.load_library()


def test_null_scene_and_arguments_are_rejected(spm):
    """Entry points validate their arguments on the host before any CUDA
    call: a null scene or a null buffer is SPM_ERR_INVALID_ARG."""
    lib = spm.load_library()
    host = np.zeros(16, np.float32)
    buf = host.ctypes.data
    assert lib.spm_compute_sequential(None, None, buf, buf) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_scene_update_sources_device(None, None, buf, buf) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_compute(None, None, buf, buf) == spm.SPM_ERR_INVALID_ARG
    assert lib.spm_query_exact(None, 1.0, 1.0, None, None) == spm.SPM_ERR_INVALID_ARG


def test_device_source_update_wants_cuda_float32(spm):
    """The binding refuses host or non-float32 tensors for the device-side
    source update before calling the library."""
    for bad in (torch.zeros(4, dtype=torch.float32), torch.zeros(4, dtype=torch.float64)):
        with pytest.raises(ValueError):
            spm.spm_scene_update_sources_device(None, None, bad, None)


def test_instrumentation_build_exports_its_readers(spm):
    """The work-counter build (a separate library; the product library
    compiles the instrumentation out) exports the device counter readers."""
    from paper_1805_08500_gb300 import build
    lib = build.build(variant="counters")
    assert lib != spm.LIB_PATH and os.path.exists(lib)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    for name in ("spm_debug_counters", "spm_debug_counters_flood", "spm_debug_counters_vertex"):
        assert f" T {name}\n" in out + "\n", name
    prod = subprocess.run(["nm", "-D", "--defined-only", spm.LIB_PATH], capture_output=True, text=True).stdout
    assert " T spm_debug_counters\n" not in prod + "\n"
