"""GPU tests of checkpoint / resume (mg_graph_export / mg_graph_import): an
imported graph is the same graph -- info, node table, mip IDs bit-exact, and
queries, propagation and lookups bit-identical to the original's -- and corrupt
or short images are rejected before anything is allocated."""
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


@pytest.mark.parametrize("dims,S", [((45, 33, 27), 40), ((64, 64, 64), 64), ((1, 1, 1), 3), ((19, 13, 11), 12)])
def test_round_trip_is_the_same_graph(mg, dims, S):
    vol = synth.make_volume(2, dims=dims, S=S) if dims != (1, 1, 1) else np.array([[[2]]], np.uint16)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), S)
    img = mg.mg_graph_export(g)
    h = mg.mg_graph_import(img.tobytes())
    for k in ("num_segments", "levels", "depth", "num_nodes", "dims", "bucket", "max_list", "pairs",
              "lut_entries"):
        assert g.info[k] == h.info[k], k
    for a, b in zip(mg.mg_graph_copy_nodes(g), mg.mg_graph_copy_nodes(h)):
        assert np.array_equal(a, b)
    for l in range(g.info["levels"]):
        assert np.array_equal(mg.mg_graph_copy_mip(g, l), mg.mg_graph_copy_mip(h, l))
    boxes = torch.from_numpy(synth.make_boxes(1, 300, dims=dims, box_max=max(dims))).cuda()
    for hist in ("u32", "f32"):
        qa = mg.mg_query_boxes(g, boxes, hist=hist).cpu().numpy()
        qb = mg.mg_query_boxes(h, boxes, hist=hist).cpu().numpy()
        assert np.array_equal(qa.view(np.uint32), qb.view(np.uint32))
    ref = oracle.box_hist(vol, S, boxes.cpu().numpy())
    assert np.array_equal(mg.mg_query_boxes(h, boxes).cpu().numpy(), ref)
    tf = torch.from_numpy(synth.make_tf(2, S, 4)).cuda()
    smp = torch.from_numpy(synth.make_samples(2, dims=dims, width=40, height=20)).cuda()
    for st in ("f32", "bf16"):
        va, vb = mg.mg_propagate_tf(g, tf, storage=st), mg.mg_propagate_tf(h, tf, storage=st)
        assert torch.equal(va, vb)
        assert torch.equal(mg.mg_render_lookup(g, va, smp), mg.mg_render_lookup(h, vb, smp))
    mg.mg_sync_status(h)
    g.close()
    h.close()


def test_corrupt_and_short_images_are_rejected(mg):
    vol = synth.make_volume(2, dims=(30, 20, 10), S=12)
    g = mg.mg_build(torch.from_numpy(vol).cuda(), 12)
    img = mg.mg_graph_export(g)
    g.close()
    for bad, status in ((img[:100], mg.MG_ERR_INVALID_ARG), (img[:-300], mg.MG_ERR_INVALID_ARG)):
        with pytest.raises(mg.MGError) as e:
            mg.mg_graph_import(bad)
        assert e.value.status == status
    wrong = img.copy()
    wrong[0] ^= 1                                  # magic
    with pytest.raises(mg.MGError) as e:
        mg.mg_graph_import(wrong)
    assert e.value.status == mg.MG_ERR_INVALID_ARG
    wrong = img.copy()
    wrong[8:12] = np.frombuffer(np.uint32(7).tobytes(), np.uint8)   # version
    with pytest.raises(mg.MGError) as e:
        mg.mg_graph_import(wrong)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
    wrong = img.copy()
    wrong[12:16] = np.frombuffer(np.uint32(13).tobytes(), np.uint8)  # S no longer fits the buckets
    with pytest.raises(mg.MGError) as e:
        mg.mg_graph_import(wrong)
    assert e.value.status == mg.MG_ERR_INVALID_ARG
    h = mg.mg_graph_import(img)                    # the intact image still loads
    h.close()
