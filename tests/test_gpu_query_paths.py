"""GPU parity of the query kernels' less common paths: many segments (the
tracked-bin flush), fp32 push with many segments, uint32 level-0 IDs, and
thin boxes that stress the per-lane block finding."""
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
def many(mg):
    vol = synth.make_volume(1, dims=(56, 48, 40), S=3000)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 3000)
    return vol, g


@pytest.mark.parametrize("chunk", [0, 96])
def test_many_segments_exact(mg, many, chunk):
    vol, g = many
    boxes = synth.make_boxes(1, Q=300, dims=(56, 48, 40), box_max=56)
    h = mg.mg_query_boxes(g, torch.from_numpy(boxes).cuda(), chunk_cubes=chunk).cpu().numpy()
    mg.mg_sync_status(g)
    assert np.array_equal(h, oracle.box_hist(vol, 3000, boxes))


def test_many_segments_fp32(mg, many):
    vol, g = many
    boxes = synth.make_boxes(1, Q=200, dims=(56, 48, 40), box_max=56)
    h = mg.mg_query_boxes(g, torch.from_numpy(boxes).cuda(), hist="f32").cpu().numpy().astype(np.float64)
    ref = oracle.box_hist(vol, 3000, boxes).astype(np.float64)
    tol = np.where(np.abs(ref) < 1e-2, 1e-7, 1e-5 * np.abs(ref))
    assert (np.abs(h - ref) <= tol).all()


def test_many_segments_plain(mg, many):
    vol, g = many
    boxes = synth.make_boxes(1, Q=60, dims=(56, 48, 40), box_max=56)
    h = mg.mg_query_boxes(g, torch.from_numpy(boxes).cuda(), schedule="plain").cpu().numpy()
    assert np.array_equal(h, oracle.box_hist(vol, 3000, boxes))


def test_uint32_level0_ids(mg):
    """More than 65536 segments: level-0 IDs stay uint32."""
    dims, S = (40, 36, 30), 70000
    rng = np.random.default_rng(7)
    vol = rng.integers(0, S, size=dims[::-1], dtype=np.uint32)
    vol[:, :, : dims[0] // 2] = 5   # some uniform area
    g = mg.mg_build(torch.from_numpy(vol.astype(np.int32)).cuda(), S)
    og = oracle.Graph(vol, S)
    assert g.N == og.N
    for level in range(og.L):
        assert (mg.mg_graph_copy_mip(g, level) == og.mip(level)).all()
    boxes = synth.make_boxes(1, Q=40, dims=dims, box_max=40)
    with pytest.raises(mg.MGError):
        mg.mg_query_boxes(g, torch.from_numpy(boxes).cuda())   # more segments than the shared histogram holds


def test_thin_boxes(mg):
    dims = (64, 64, 64)
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 64)
    rng = np.random.default_rng(9)
    boxes = []
    for _ in range(400):
        side = [int(rng.integers(1, 65)) for _ in range(3)]
        side[int(rng.integers(0, 3))] = int(rng.integers(1, 3))   # one thin axis
        o = [int(rng.integers(0, 64 - s + 1)) for s in side]
        boxes.append(o + side)
    boxes = np.array(boxes, np.int32)
    for chunk in (0, 33, 1000):
        h = mg.mg_query_boxes(g, torch.from_numpy(boxes).cuda(), chunk_cubes=chunk).cpu().numpy()
        assert np.array_equal(h, oracle.box_hist(vol, 64, boxes)), chunk
