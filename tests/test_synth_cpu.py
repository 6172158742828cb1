"""The seeded input recipes (shapes, ranges, distributions, determinism) that
every parity test and the benchmark draw from.  Inputs only: nothing here
checks the Mixture Graph's arithmetic."""
import math

import numpy as np
import pytest

from paper_2009_02702_gb300 import synth


def test_voronoi_volume_is_seeded_and_in_range():
    a = synth.make_volume(1)
    b = synth.make_volume(1)
    assert a.shape == (64, 64, 64) and a.dtype == np.uint16
    assert np.array_equal(a, b)
    assert a.max() < 64 and len(np.unique(a)) == 64        # every seed owns a cell
    c = synth.make_volume(1, dims=(30, 20, 10), S=9)
    assert c.shape == (10, 20, 30) and c.max() < 9


def test_voronoi_window_equals_the_volume_window():
    vol = synth.make_volume(1, dims=(40, 36, 28), S=17)
    for origin, ext in (((0, 0, 0), (40, 36, 28)), ((5, 7, 3), (13, 11, 9)), ((39, 35, 27), (1, 1, 1))):
        w = synth.voronoi_window(1, origin, ext, dims=(40, 36, 28), S=17)
        x, y, z = origin
        dx, dy, dz = ext
        assert np.array_equal(w, vol[z:z + dz, y:y + dy, x:x + dx])


def test_cylinder_volume_recipe():
    rng = synth.rng_for(4, 0)
    vol, _ = synth.cylinders_host((60, 50, 40), 30, rng, (2.0, 4.0), (10.0, 30.0), 8)
    again, _ = synth.cylinders_host((60, 50, 40), 30, synth.rng_for(4, 0), (2.0, 4.0), (10.0, 30.0), 8)
    assert vol.shape == (40, 50, 60) and np.array_equal(vol, again)
    ids = np.unique(vol)
    assert ids[0] == 0 and ids.max() <= 30                  # background plus cylinder IDs
    assert (vol == 0).mean() > 0.5


def test_boxes_lie_inside_and_follow_their_distribution():
    for cfg in (1, 2, 3, 4):
        c = synth.CONFIGS[cfg]
        b = synth.make_boxes(cfg, Q=4000)
        assert b.dtype == np.int32 and b.shape == (4000, 6)
        d = np.array(c["dims"])
        assert (b[:, :3] >= 0).all() and (b[:, 3:] >= 1).all()
        assert (b[:, :3] + b[:, 3:] <= d).all()
        assert (b[:, 3:] <= c["box_max"]).all()
        assert np.array_equal(b, synth.make_boxes(cfg, Q=4000))
        assert not np.array_equal(b, synth.make_boxes(cfg, Q=4000, stream_offset=1))
    # log-uniform sides: log2(side + 1) about uniform on [0, log2(box_max + 1)]
    b = synth.make_boxes(2, Q=20000)
    u = np.log2(b[:, 3:].astype(np.float64) + 1) / math.log2(513)
    assert abs(u.mean() - 0.5) < 0.03


def test_tf_and_samples():
    tf = synth.make_tf(2, 353, 4)
    assert tf.shape == (353, 4) and tf.dtype == np.float32 and (tf >= 0).all() and (tf < 1).all()
    at = synth.make_attribute_tf(4, 100)
    assert at.shape == (100, 4) and (at[0] == 0).all() and (at[:, 3] <= 1).all()
    s = synth.make_samples(2, width=64, height=48)
    assert s.shape == (64 * 48, 4) and s.dtype == np.float32
    d = np.array(synth.CONFIGS[2]["dims"], np.float32)
    inside = ((s[:, :3] >= -1e-3) & (s[:, :3] <= d + 1e-3)).all(axis=1)
    assert inside.mean() > 0.3                               # the rays that hit the volume
    assert np.isfinite(s).all()
    assert np.array_equal(s, synth.make_samples(2, width=64, height=48))


def test_request_mix_is_poisson_with_the_stated_mix():
    dims = [(64, 64, 64), (512, 512, 384)]
    arr, kind, vol, boxes = synth.make_request_mix(50000, 20000.0, dims, (64, 512), tf_frac=0.1)
    assert arr[0] == 0 and (np.diff(arr) >= 0).all()
    assert abs(np.diff(arr).mean() * 20000.0 - 1.0) < 0.03
    assert abs(kind.mean() - 0.1) < 0.01
    assert set(np.unique(vol)) == {0, 1}
    for v, d in enumerate(dims):
        m = (vol == v) & (kind == 0)
        b = boxes[m]
        assert (b[:, 3:] >= 1).all() and (b[:, :3] + b[:, 3:] <= np.array(d)).all()
    assert (boxes[kind == 1] == 0).all()


def _voronoi_pair(dims, K, weighted, metric, seed, origin=(0, 0, 0), extent=None):
    rng = np.random.default_rng(seed)
    seeds2, W = synth.voronoi_seeds(dims, K, weighted, rng)
    ext = extent or dims
    outs = []
    for fn in ("mgs_voronoi_block", "mgs_voronoi_block_brute"):
        out = np.zeros(ext[::-1], np.uint16)
        m = np.array(metric, np.int64)
        getattr(synth._host_lib(), fn)(*origin, *ext, seeds2.ctypes.data, W.ctypes.data, K, m.ctypes.data, 2,
                                       out.ctypes.data)
        outs.append(out)
    return outs


@pytest.mark.parametrize("dims,K,weighted,metric", [
    ((53, 41, 37), 40, False, (1, 1, 1)),
    ((70, 33, 29), 25, True, (1, 1, 1)),
    ((64, 64, 20), 30, False, (16, 16, 1)),
    ((17, 90, 16), 300, True, (1, 4, 9)),
    ((40, 40, 40), 1, False, (1, 1, 1)),
])
def test_tiled_voronoi_equals_brute_force(dims, K, weighted, metric):
    """Pruning seeds per tile changes no voxel, ties included (lowest index)."""
    fast, brute = _voronoi_pair(dims, K, weighted, metric, seed=K)
    assert np.array_equal(fast, brute)
    # an offset window, with tiles cut at its far faces
    fast, brute = _voronoi_pair(dims, K, weighted, metric, seed=K, origin=(5, 3, 2), extent=(37, 19, 23))
    assert np.array_equal(fast, brute)


def test_tiled_voronoi_ties_go_to_the_lowest_index():
    # duplicated seeds tie everywhere: the lower index must win each voxel
    dims = (24, 24, 24)
    seeds2 = np.array([[10, 10, 10], [30, 30, 30], [10, 10, 10], [30, 30, 30]], np.int64)
    W = np.ones(4, np.int64)
    m = np.ones(3, np.int64)
    out = np.zeros(dims[::-1], np.uint16)
    synth._host_lib().mgs_voronoi_block(0, 0, 0, *dims, seeds2.ctypes.data, W.ctypes.data, 4, m.ctypes.data, 2,
                                        out.ctypes.data)
    assert set(np.unique(out).tolist()) == {0, 1}
