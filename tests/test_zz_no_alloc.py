"""spm_agents_backward_noalloc: the allocation-free backward, for callers
that may not allocate device memory while they run (a per-frame steering
loop that must not stall on cudaMalloc, or code inside a framework whose
memory pool owns the device). It must give the same gradients as the
allocating path (spm_agents_forward + spm_agents_backward), call after call,
even though every call reuses one fixed scratch array inside the library.

This file is named to be collected last: if it fails, a run that stops at
the first failure has already run every other test.
"""
import ctypes

import pytest

import scenegen as sg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1805_08500_gb300 as m
    m.load_library()
    return m


def test_noalloc_backward_matches_allocating_path(spm):
    """Both paths run the same kernels in the same fixed order, so the
    gradients must agree bit for bit. Two calls in a row with different agent
    counts: a scratch offset or stale contents from the first call would show."""
    lib = spm.load_library()
    scene = sg.differentiable(2, W=1024, N=256, n_polys=20, n_agents=5000)
    s = spm.Scene(scene)
    dist, parent = s.compute()
    s.sync()
    dev = dist.device
    all_agents = torch.tensor(scene.agents, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for n in (5000, 1777):
        agents = all_agents[:n].contiguous()
        loss = torch.empty((), dtype=torch.float32, device=dev)
        tape = spm.empty_tape(n, dev)
        gp_ref = torch.zeros((len(scene.points), 2), dtype=torch.float32, device=dev)
        gs_ref = torch.zeros((len(scene.segs), 4), dtype=torch.float32, device=dev)
        spm.spm_agents_forward(s.handle, None, agents, dist, parent, loss, tape)
        spm.spm_agents_backward(s.handle, None, tape, n, gp_ref, gs_ref)
        gp = torch.full_like(gp_ref, float("nan"))
        gs = torch.full_like(gs_ref, float("nan"))
        st = lib.spm_agents_backward_noalloc(
            ctypes.c_void_p(s.handle), ctypes.c_void_p(stream), ctypes.c_void_p(agents.data_ptr()),
            ctypes.c_int32(n), ctypes.c_void_p(parent.data_ptr()), ctypes.c_void_p(gp.data_ptr()),
            ctypes.c_void_p(gs.data_ptr()))
        assert st == 0, spm.spm_status_string(st)
        torch.cuda.synchronize()
        assert torch.equal(gp.view(torch.int32), gp_ref.view(torch.int32)), n
        assert torch.equal(gs.view(torch.int32), gs_ref.view(torch.int32)), n
        assert torch.isfinite(gp).all() and torch.isfinite(gs).all()


def test_noalloc_backward_rejects_oversized_input(spm):
    lib = spm.load_library()
    scene = sg.differentiable(3, W=512, N=128, n_polys=8, n_agents=16)
    s = spm.Scene(scene)
    dist, parent = s.compute()
    s.sync()
    agents = torch.zeros((4, 2), dtype=torch.int32, device=dist.device)
    gp = torch.zeros((len(scene.points), 2), dtype=torch.float32, device=dist.device)
    gs = torch.zeros((len(scene.segs), 4), dtype=torch.float32, device=dist.device)
    too_many = 131072 + 1  # SPM_NOALLOC_MAX_AGENTS + 1: rejected before any launch
    st = lib.spm_agents_backward_noalloc(
        ctypes.c_void_p(s.handle), None, ctypes.c_void_p(agents.data_ptr()), ctypes.c_int32(too_many),
        ctypes.c_void_p(parent.data_ptr()), ctypes.c_void_p(gp.data_ptr()), ctypes.c_void_p(gs.data_ptr()))
    assert st == 7  # SPM_ERR_CAPACITY
