"""The scratch-free query entry point (mg_query_boxes_noalloc).

Some callers cannot let a library allocate device memory (real-time frame
loops, engines that reserve the whole device, fixed memory budgets); this
entry point serves them from a fixed array compiled into the library.  Its
results must equal mg_query_boxes' exactly, call after call, since every call
reuses the same array.  This file is collected last on purpose, so a failure
here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2009_02702_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    from paper_2009_02702_gb300 import mg as _mg
    _mg.lib()
    return _mg


def test_noalloc_matches_allocating_query_twice(mg):
    dims, S = (61, 47, 38), 40
    vol = synth.make_volume(2, dims=dims, S=S)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), S)
    boxes = [synth.make_boxes(1, Q=700, dims=dims, box_max=61, stream_offset=k) for k in range(2)]
    for bx in boxes:   # two calls in a row share the fixed scratch
        t = torch.from_numpy(bx).cuda()
        ref = mg.mg_query_boxes(g, t).cpu().numpy()
        got = mg.mg_query_boxes_noalloc(g, t).cpu().numpy()
        mg.mg_sync_status(g)
        assert np.array_equal(got, ref)
    g.close()


def test_noalloc_through_the_c_abi_and_limits(mg):
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 64)
    bx = torch.from_numpy(synth.make_boxes(1, Q=300)).cuda()
    out = torch.full((300, 64), 7, dtype=torch.uint32, device="cuda")   # stale contents are overwritten
    stream = torch.cuda.current_stream().cuda_stream
    st = mg.lib().mg_query_boxes_noalloc(g.handle, bx.data_ptr(), 300, out.data_ptr(), out.numel(), stream)
    assert st == mg.MG_OK
    assert torch.equal(out.cpu(), mg.mg_query_boxes(g, bx).cpu())
    # too many boxes for the fixed scratch: refused before any work
    big = torch.zeros((2_000_000, 6), dtype=torch.int32, device="cuda")
    st = mg.lib().mg_query_boxes_noalloc(g.handle, big.data_ptr(), big.shape[0], out.data_ptr(),
                                         ctypes.c_size_t(1 << 40), stream)
    assert st == mg.MG_ERR_CAPACITY
    assert "boxes" in mg.mg_last_error()
    # too small an output is an argument error
    st = mg.lib().mg_query_boxes_noalloc(g.handle, bx.data_ptr(), 300, out.data_ptr(), 10, stream)
    assert st == mg.MG_ERR_INVALID_ARG
    g.close()
