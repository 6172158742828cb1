"""The scratch-free query entry point (mg_query_boxes_noalloc).

Some callers cannot let a library allocate device memory (real-time frame
loops, engines that reserve the whole device, fixed memory budgets); this
entry point serves them from a fixed array compiled into the library.  Its
results must equal the brute-force counts of the oracle and mg_query_boxes'
exactly, call after call, since every call reuses the same array.  This file
is collected last on purpose, so a failure here leaves every other test
already run.
"""
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
        assert np.array_equal(got, oracle.box_hist(vol, S, bx))
    g.close()


def test_noalloc_through_the_c_abi_and_limits(mg):
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 64)
    bx_h = synth.make_boxes(1, Q=300)
    bx = torch.from_numpy(bx_h).cuda()
    out = torch.full((300, 64), 7, dtype=torch.uint32, device="cuda")   # stale contents are overwritten
    stream = torch.cuda.current_stream().cuda_stream
    st = mg.lib().mg_query_boxes_noalloc(g.handle, bx.data_ptr(), 300, out.data_ptr(), out.numel(), stream)
    assert st == mg.MG_OK
    assert np.array_equal(out.cpu().numpy(), oracle.box_hist(vol, 64, bx_h))
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


def test_noalloc_more_boxes_than_one_scan_block(mg):
    # 300,000 boxes: the offsets take the device-wide scan, whose partial sums
    # also come out of the fixed array
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 64)
    Q = 300_000
    rng = np.random.default_rng(31)
    bx_h = np.concatenate([rng.integers(0, 63, (Q, 3)), rng.integers(1, 3, (Q, 3))], 1).astype(np.int32)
    got = mg.mg_query_boxes_noalloc(g, torch.from_numpy(bx_h).cuda()).cpu().numpy()
    mg.mg_sync_status(g)
    assert np.array_equal(got, oracle.box_hist(vol, 64, bx_h))
    g.close()


def test_noalloc_footprint_too_large_leaves_output(mg):
    # 1,500 boxes with odd origins on a 512x512x384 volume need about 75 MiB
    # of footprint blocks and chunks: more than the fixed array holds, so the
    # call is refused with the output left as it was
    c = synth.CONFIGS[2]
    g = mg.mg_build(synth.make_volume(2, device="cuda"), c["S"])
    Q = 1500
    bx = torch.tensor([[1, 1, 1, 510, 510, 382]] * Q, dtype=torch.int32, device="cuda")
    out = torch.full((Q, c["S"]), 5, dtype=torch.uint32, device="cuda")
    with pytest.raises(mg.MGError) as e:
        mg.mg_query_boxes_noalloc(g, bx, out=out)
    assert e.value.status == mg.MG_ERR_CAPACITY
    assert "split the batch" in str(e.value)
    torch.cuda.synchronize()
    assert bool((out == 5).all())
    # a batch that fits still succeeds right after the refusal
    small = bx[:8].contiguous()
    got = mg.mg_query_boxes_noalloc(g, small).cpu().numpy()
    ref = mg.mg_query_boxes(g, small).cpu().numpy()
    mg.mg_sync_status(g)
    assert np.array_equal(got, ref)
    assert (got.astype(np.int64).sum(axis=1) == 510 * 510 * 382).all()
    g.close()
