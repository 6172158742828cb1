"""Failure handling on the GPU without faulting or hanging it.

A bounded device wait that runs out (a flag nothing sets) reports
MG_ERR_TIMEOUT and leaves the context usable; an allocator that returns NULL
(failure injected on the host) makes the build return MG_ERR_OOM, after which
normal calls still work."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2009_02702_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    from paper_2009_02702_gb300 import mg as _mg
    _mg.lib()
    return _mg


def _graph_works(mg):
    vol = synth.make_volume(1, dims=(20, 18, 16), S=10)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 10)
    tf = synth.make_tf(1, 10, 4)
    vals = mg.mg_propagate_tf(g, torch.from_numpy(tf).cuda()).cpu().numpy()
    mg.mg_sync_status(g)
    og = oracle.Graph(vol, 10)
    ref = oracle.propagate(og.p, og.q, og.a, og.b, 10, tf)
    g.close()
    return np.allclose(vals, ref, rtol=1e-5, atol=1e-7)


def test_bounded_wait_times_out_and_gpu_stays_usable(mg):
    assert mg.mg_selftest_bounded_wait(True) == mg.MG_OK
    assert mg.mg_selftest_bounded_wait(False, 1 << 14) == mg.MG_ERR_TIMEOUT
    assert mg.mg_selftest_bounded_wait(False, 1) == mg.MG_ERR_TIMEOUT
    assert mg.mg_selftest_bounded_wait(True, 1) == mg.MG_OK
    with pytest.raises(mg.MGError):
        mg.mg_selftest_bounded_wait(False, 0)
    torch.cuda.synchronize()
    assert _graph_works(mg)


def test_allocator_returning_null_gives_oom(mg):
    vol = synth.make_volume(1, dims=(24, 20, 18), S=12)
    ids = torch.from_numpy(vol).cuda()
    lib = mg.lib()
    outcomes = []
    for budget in (0, 1, 2, 5, 9, 14, 1 << 30):
        calls = {"n": 0}
        live = {}

        def alloc(ctx, nbytes, stream):
            calls["n"] += 1
            if calls["n"] > budget:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
            live[p] = True
            return p

        def free(ctx, ptr, nbytes, stream):
            if live.pop(int(ptr), None):
                torch.cuda.caching_allocator_delete(int(ptr))

        a = mg.mg_allocator(None, mg.ALLOC_FN(alloc), mg.FREE_FN(free))
        h = ctypes.c_void_p()
        nz, ny, nx = ids.shape
        st = lib.mg_build(ids.data_ptr(), nx, ny, nz, 12, ctypes.byref(mg.mg_build_opts(2)), ctypes.byref(a),
                          torch.cuda.current_stream().cuda_stream, ctypes.byref(h))
        torch.cuda.synchronize()
        outcomes.append(st)
        if st == mg.MG_OK:
            lib.mg_free(h.value)
        else:
            assert st == mg.MG_ERR_OOM, (budget, st, mg.mg_last_error())
            assert h.value is None
        torch.cuda.synchronize()
        assert not live, (budget, len(live))   # everything handed out was given back
    assert outcomes[0] == mg.MG_ERR_OOM and outcomes[-1] == mg.MG_OK
    assert _graph_works(mg)


def test_misaligned_allocator_is_refused(mg):
    # an allocator whose pointers are not 256-byte aligned is refused before
    # any kernel reads through them; everything handed out is given back
    vol = synth.make_volume(1, dims=(24, 20, 18), S=12)
    ids = torch.from_numpy(vol).cuda()
    lib = mg.lib()
    live = {}

    def alloc(ctx, nbytes, stream):
        p = torch.cuda.caching_allocator_alloc(int(nbytes) + 256, 0, int(stream or 0))
        live[p + 16] = p
        return p + 16

    def free(ctx, ptr, nbytes, stream):
        p = live.pop(int(ptr), None)
        if p is not None:
            torch.cuda.caching_allocator_delete(p)

    a = mg.mg_allocator(None, mg.ALLOC_FN(alloc), mg.FREE_FN(free))
    h = ctypes.c_void_p()
    nz, ny, nx = ids.shape
    st = lib.mg_build(ids.data_ptr(), nx, ny, nz, 12, ctypes.byref(mg.mg_build_opts(2)), ctypes.byref(a),
                      torch.cuda.current_stream().cuda_stream, ctypes.byref(h))
    torch.cuda.synchronize()
    assert st == mg.MG_ERR_INVALID_ARG and h.value is None
    assert "256-byte" in mg.mg_last_error()
    assert not live
    assert _graph_works(mg)
