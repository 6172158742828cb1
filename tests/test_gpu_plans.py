"""GPU parity of the captured query plans, the autotuner and the naive
brute-force schedule against the CPU oracle."""
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


@pytest.fixture(scope="module")
def cfg1(mg):
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 64)
    return vol, g


def test_plan_u32_matches_oracle_for_varying_batches(mg, cfg1):
    vol, g = cfg1
    plan = mg.QueryPlan(g, max_Q=800)
    for k, Q in enumerate([800, 1, 333, 800, 57]):
        boxes = synth.make_boxes(1, Q=Q, stream_offset=k)
        h = plan.run(torch.from_numpy(boxes).cuda()).cpu().numpy()
        mg.mg_sync_status(g)
        assert np.array_equal(h, oracle.box_hist(vol, 64, boxes)), Q
    assert plan.run(torch.zeros((0, 6), dtype=torch.int32, device="cuda")).shape == (0, 64)
    plan.close()


def test_plan_many_tiles_partial_tiles_and_timing(mg, cfg1):
    # hundreds of 16-box tiles chained by the plan's single-pass scan, a
    # partial last tile, and a malformed box in the middle of the batch
    vol, g = cfg1
    plan = mg.QueryPlan(g, max_Q=6000, timing=True)
    for k, Q in enumerate([6000, 4999, 17]):
        boxes = synth.make_boxes(1, Q=Q, stream_offset=10 + k)
        h = plan.run(torch.from_numpy(boxes).cuda()).cpu().numpy()
        mg.mg_sync_status(g)
        assert np.array_equal(h, oracle.box_hist(vol, 64, boxes)), Q
        plan_ms, main_ms = plan.timing()
        assert plan_ms > 0 and main_ms > 0
    boxes = synth.make_boxes(1, Q=3000, stream_offset=20)
    bad = boxes.copy()
    bad[1234, 3] = 0   # empty extent
    h = plan.run(torch.from_numpy(bad).cuda()).cpu().numpy()
    with pytest.raises(mg.MGError) as e:
        mg.mg_sync_status(g)
    assert e.value.status == mg.MG_ERR_INVALID_ARG   # the device saw a malformed box
    ref = oracle.box_hist(vol, 64, boxes)
    keep = np.arange(3000) != 1234
    assert np.array_equal(h[keep], ref[keep]) and (h[1234] == 0).all()
    plan.close()
    untimed = mg.QueryPlan(g, max_Q=10)
    untimed.run(torch.from_numpy(synth.make_boxes(1, Q=10)).cuda())
    with pytest.raises(mg.MGError) as e:
        untimed.timing()
    assert e.value.status == mg.MG_ERR_INVALID_ARG
    untimed.close()


@pytest.mark.parametrize("hist", ["u32", "f32"])
def test_plan_runs_on_unaligned_caller_buffers(mg, cfg1, hist):
    # the plan reads the boxes from and accumulates into the caller's buffers;
    # views one element past a 16-byte boundary exercise the zeroing's ends
    vol, g = cfg1
    Q = 700
    boxes = synth.make_boxes(1, Q=Q, stream_offset=40)
    dt = torch.uint32 if hist == "u32" else torch.float32
    plan = mg.QueryPlan(g, max_Q=Q, hist=hist)
    bflat = torch.empty(Q * 6 + 1, dtype=torch.int32, device="cuda")
    bview = bflat[1:].view(Q, 6)
    bview.copy_(torch.from_numpy(boxes))
    oflat = torch.full((Q * 64 + 3,), 7, dtype=dt, device="cuda")
    oview = oflat[1:1 + Q * 64].view(Q, 64)
    plan.run(bview, out=oview)
    mg.mg_sync_status(g)
    ref = oracle.box_hist(vol, 64, boxes)
    assert np.array_equal(oview.cpu().numpy().astype(np.int64), ref.astype(np.int64))
    # nothing outside the output rows is touched
    assert oflat[0].item() == 7 and (oflat[1 + Q * 64:] == 7).all().item()
    plan.close()


@pytest.mark.parametrize("chunk", [1000, 3, 65536])
def test_plan_non_power_of_two_and_extreme_chunks(mg, cfg1, chunk):
    # chunk maps by division (non powers of two) and by shift, tiny and huge chunks
    vol, g = cfg1
    boxes = synth.make_boxes(1, Q=500, stream_offset=50)
    plan = mg.QueryPlan(g, max_Q=500, chunk_cubes=chunk, max_chunks=500 * 4096)
    h = plan.run(torch.from_numpy(boxes).cuda()).cpu().numpy()
    mg.mg_sync_status(g)
    assert np.array_equal(h, oracle.box_hist(vol, 64, boxes))
    plan.close()


def test_plan_long_lookback_chain(mg, cfg1):
    # 6,250 tiles chained by the look-back of the single-pass scan
    vol, g = cfg1
    boxes = synth.make_boxes(1, Q=100000, stream_offset=30)
    plan = mg.QueryPlan(g, max_Q=100000)
    h = plan.run(torch.from_numpy(boxes).cuda()).cpu().numpy()
    mg.mg_sync_status(g)
    assert np.array_equal(h, oracle.box_hist(vol, 64, boxes))
    plan.close()


def test_plan_fp32_and_bf16(mg, cfg1):
    vol, g = cfg1
    boxes = synth.make_boxes(1, Q=300)
    ref = oracle.box_hist(vol, 64, boxes).astype(np.float64)
    for alpha, rtol in (("f32", 1e-5), ("bf16", None)):
        plan = mg.QueryPlan(g, max_Q=300, hist="f32", alpha=alpha)
        h = plan.run(torch.from_numpy(boxes).cuda()).cpu().numpy().astype(np.float64)
        direct = mg.mg_query_boxes(g, torch.from_numpy(boxes).cuda(), hist="f32", alpha=alpha).cpu().numpy()
        assert np.allclose(h, direct, rtol=1e-6, atol=1e-3)
        if rtol:
            tol = np.where(np.abs(ref) < 1e-2, 1e-7, rtol * np.abs(ref))
            assert (np.abs(h - ref) <= tol).all()
        plan.close()


def test_plan_capacity_overflow_is_reported(mg, cfg1):
    vol, g = cfg1
    plan = mg.QueryPlan(g, max_Q=100, max_blocks=10, max_chunks=10)
    boxes = synth.make_boxes(1, Q=100)
    h = plan.run(torch.from_numpy(boxes).cuda()).cpu().numpy()
    with pytest.raises(mg.MGError) as e:
        mg.mg_sync_status(g)
    assert e.value.status == mg.MG_ERR_CAPACITY
    assert (h == 0).all()
    plan.close()


def test_autotune_and_cache(mg, cfg1, tmp_path):
    vol, g = cfg1
    boxes = torch.from_numpy(synth.make_boxes(1, Q=500)).cuda()
    cache = str(tmp_path / "tune.json")
    r = mg.mg_query_autotune(g, boxes, cache=cache, key="cfg1")
    assert r["chunk_cubes"] in (1024, 2048, 4096, 8192, 16384) and r["block_threads"] in (128, 256, 512)
    assert not r["cached"]
    r2 = mg.mg_query_autotune(g, boxes, cache=cache, key="cfg1")
    assert r2["cached"] and r2["chunk_cubes"] == r["chunk_cubes"]
    h = mg.mg_query_boxes(g, boxes).cpu().numpy()   # uses the tuned shape
    assert np.array_equal(h, oracle.box_hist(vol, 64, boxes.cpu().numpy()))


@pytest.mark.parametrize("hist", ["u32", "f32"])
def test_naive_schedule(mg, cfg1, hist):
    vol, g = cfg1
    boxes = synth.make_boxes(1, Q=200)
    h = mg.mg_query_boxes(g, torch.from_numpy(boxes).cuda(), schedule="naive", hist=hist).cpu().numpy()
    assert np.array_equal(h.astype(np.int64), oracle.box_hist(vol, 64, boxes).astype(np.int64))
