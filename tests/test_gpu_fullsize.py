"""Parity at the full workload sizes, in the launch configuration bench.py
times (autotuned launch shape, captured query plan).

The oracle cannot redo a whole batch at these sizes, so every output is
checked two ways: a property that holds at any size (each u32 histogram sums
to its clipped box volume, exactly, for every box of the batch) and sampled
outputs the oracle computes one by one -- box histograms by brute-force
counting over the box's voxels, and voxel / ray-sample colours as the direct
fp64 sum over the voxel's footprint (Sec. 3.4).  The oracle's voxels come
from the host generators (a window of the volume, or the whole volume), never
from the GPU.  Besides the sampled boxes, the ten largest boxes of every batch
and whole-volume boxes appended to it are compared element by element with
the oracle's brute-force counts over the host volume.
"""
import numpy as np
import pytest

import oracle
from paper_2009_02702_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL, ATOL_SMALL = 1e-5, 1e-7


def fp32_close(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = np.where(np.abs(ref) < 1e-2, ATOL_SMALL, RTOL * np.abs(ref))
    ok = (np.abs(x - ref) <= tol) & ((ref != 0) | (x == 0))
    return bool(ok.all()), float(np.max(np.abs(x - ref)) if x.size else 0.0)


@pytest.fixture(scope="module")
def mg():
    from paper_2009_02702_gb300 import mg as _mg
    _mg.lib()
    return _mg


def clipped(boxes, dims):
    d = np.array(dims, np.int64)
    lo = boxes[:, :3].astype(np.int64)
    hi = np.minimum(lo + boxes[:, 3:].astype(np.int64), d[None, :])
    return lo, hi - lo


def sample_boxes(boxes, dims, n, max_voxels, seed):
    """Seeded pick of n boxes whose clipped volume the host can count quickly,
    spread over the size range."""
    _, side = clipped(boxes, dims)
    vol = side.prod(axis=1)
    cand = np.flatnonzero(vol <= max_voxels)
    order = cand[np.argsort(vol[cand], kind="stable")]
    pick = order[np.linspace(0, len(order) - 1, n).astype(np.int64)]
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([pick, rng.choice(cand, size=n // 2, replace=False)]))


class Windows:
    """Host voxels of a box: a window generated on the host (Voronoi) or cut
    from the host volume."""

    def __init__(self, cfg, vol_h=None):
        self.cfg, self.vol_h = cfg, vol_h

    def block(self, origin, side):
        if self.vol_h is not None:
            x, y, z = origin
            return self.vol_h[z:z + side[2], y:y + side[1], x:x + side[0]]
        return synth.voronoi_window(self.cfg, origin, side)

    def hist(self, origin, side, S):
        b = np.ascontiguousarray(self.block(origin, side))
        return oracle.box_hist(b, S, np.array([[0, 0, 0, side[0], side[1], side[2]]], np.int32))[0]


def run_plan(mg, g, boxes_d, hist, key, alpha="f32"):
    """The bench's query launch: autotune on the batch, then one plan run."""
    mg.mg_query_autotune(g, boxes_d, hist=hist, alpha=alpha, key=key)
    plan = mg.QueryPlan(g, max_Q=boxes_d.shape[0], hist=hist, alpha=alpha)
    out = plan.run(boxes_d)
    mg.mg_sync_status(g)
    res = out.cpu().numpy()
    plan.close()
    return res


def largest_boxes(boxes, dims, k, extra=0):
    """The k boxes of the batch with the largest clipped volume, plus the last
    `extra` rows (boxes appended to the batch)."""
    _, side = clipped(boxes, dims)
    body = len(boxes) - extra
    big = np.argsort(side[:body].prod(axis=1), kind="stable")[::-1][:k]
    return np.concatenate([big, np.arange(body, len(boxes))])


def check_counts(h, boxes, dims, win, S, n, max_voxels, seed, vol_h=None, extra=0):
    _, side = clipped(boxes, dims)
    sums = h.astype(np.uint64).sum(axis=1)
    assert np.array_equal(sums, side.prod(axis=1).astype(np.uint64))
    for i in sample_boxes(boxes, dims, n, max_voxels, seed):
        ref = win.hist(boxes[i, :3], side[i], S)
        assert np.array_equal(h[i], ref), i
    if vol_h is not None:
        # the largest footprints (highest mip levels, longest run lists) and
        # the appended whole-volume boxes, element by element
        idx = largest_boxes(boxes, dims, 10, extra)
        ref = oracle.box_hist(vol_h, S, boxes[idx])
        for k, i in enumerate(idx):
            assert np.array_equal(h[i], ref[k]), (int(i), boxes[i].tolist())


def voxel_colour_checks(mg, g, vals, win, tf, dims, S, levels, per_level, seed, check):
    """Interior voxels of the given levels: GPU colour vs the fp64 direct sum."""
    rng = np.random.default_rng(seed)
    tf64 = tf.astype(np.float64)
    for l in levels:
        e = 1 << l
        if any(d // e < 1 for d in dims):
            continue
        mip = mg.mg_graph_copy_mip(g, l)
        for _ in range(per_level):
            X, Y, Z = (int(rng.integers(0, d // e)) for d in dims)
            blk = win.block((X * e, Y * e, Z * e), (e, e, e))
            ref = np.bincount(blk.ravel(), minlength=S).astype(np.float64) @ tf64 / blk.size
            check(vals[mip[Z, Y, X]], ref, (l, X, Y, Z))


def sample_colour_checks(mg, g, look, samples, vals_dims, win, tf, S, n, seed, check, max_level=7):
    """Ray samples whose selected voxel is interior and at most 2^max_level
    wide: GPU lookup vs the fp64 direct sum of that voxel."""
    dims = oracle.level_dims(*vals_dims)
    lev, vox = oracle.sample_voxels(dims, samples)
    rng = np.random.default_rng(seed)
    idx = rng.permutation(samples.shape[0])
    tf64 = tf.astype(np.float64)
    done = 0
    for i in idx:
        l = int(lev[i])
        if l > max_level:
            continue
        nx, ny, nz = (int(v) for v in dims[l])
        v = int(vox[i])
        X, Y, Z = v % nx, (v // nx) % ny, v // (nx * ny)
        e = 1 << l
        if (X + 1) * e > vals_dims[0] or (Y + 1) * e > vals_dims[1] or (Z + 1) * e > vals_dims[2]:
            continue
        blk = win.block((X * e, Y * e, Z * e), (e, e, e))
        ref = np.bincount(blk.ravel(), minlength=S).astype(np.float64) @ tf64 / blk.size
        check(look[i], ref, (i, l))
        done += 1
        if done >= n:
            break
    assert done >= n // 2


def fp32_check(x, ref, where):
    ok, err = fp32_close(x, ref)
    assert ok, (where, err)


# ---------------------------------------------------------------------------
# config 2: 512x512x384, 353 segments, 10,000 boxes (the bench workload)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg2(mg):
    c = synth.CONFIGS[2]
    g = mg.mg_build(synth.make_volume(2, device="cuda"), c["S"])
    yield g, c
    g.close()


@pytest.fixture(scope="module")
def vol2():
    return synth.make_volume(2)


def with_whole_volume(boxes, dims):
    """The batch with two boxes appended: the whole volume, and the volume
    less one voxel on every face (odd origins: runs rise and fall on every
    axis)."""
    nx, ny, nz = dims
    extra = np.array([[0, 0, 0, nx, ny, nz], [1, 1, 1, nx - 2, ny - 2, nz - 2]], np.int32)
    return np.ascontiguousarray(np.concatenate([boxes, extra])), len(extra)


def test_cfg2_full_batch_u32_exact(mg, cfg2, vol2):
    g, c = cfg2
    boxes, extra = with_whole_volume(synth.make_boxes(2), c["dims"])
    h = run_plan(mg, g, torch.from_numpy(boxes).cuda(), "u32", c["name"])
    check_counts(h, boxes, c["dims"], Windows(2, vol2), c["S"], 40, 1 << 21, 1, vol_h=vol2, extra=extra)


def test_cfg2_full_batch_f32_within_tolerance(mg, cfg2, vol2):
    g, c = cfg2
    boxes, extra = with_whole_volume(synth.make_boxes(2), c["dims"])
    h = run_plan(mg, g, torch.from_numpy(boxes).cuda(), "f32", c["name"])
    _, side = clipped(boxes, c["dims"])
    assert np.allclose(h.astype(np.float64).sum(axis=1), side.prod(axis=1), rtol=1e-5)
    win = Windows(2, vol2)
    for i in sample_boxes(boxes, c["dims"], 24, 1 << 21, 2):
        ok, err = fp32_close(h[i], win.hist(boxes[i, :3], side[i], c["S"]))
        assert ok, (i, err)
    idx = largest_boxes(boxes, c["dims"], 10, extra)
    ref = oracle.box_hist(vol2, c["S"], boxes[idx])
    for k, i in enumerate(idx):
        ok, err = fp32_close(h[i], ref[k])
        assert ok, (int(i), err)


def test_cfg2_propagate_and_frame(mg, cfg2, vol2):
    g, c = cfg2
    tf = synth.make_tf(2, c["S"], 4)
    vals_d = mg.mg_propagate_tf(g, torch.from_numpy(tf).cuda())
    samples = synth.make_samples(2)
    look = mg.mg_render_lookup(g, vals_d, torch.from_numpy(samples).cuda()).cpu().numpy()
    mg.mg_sync_status(g)
    vals = vals_d.cpu().numpy()
    win = Windows(2, vol2)
    voxel_colour_checks(mg, g, vals, win, tf, c["dims"], c["S"], (0, 1, 3, 5, 7), 12, 3, fp32_check)
    sample_colour_checks(mg, g, look, samples, c["dims"], win, tf, c["S"], 120, 4, fp32_check)


# ---------------------------------------------------------------------------
# config 3: 2048x2048x300, 1,182 segments, 100,000 boxes; fp16 weights
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg3(mg):
    c = synth.CONFIGS[3]
    g = mg.mg_build(synth.make_volume(3, device="cuda"), c["S"])
    yield g, c
    g.close()


@pytest.fixture(scope="module")
def vol3():
    return synth.make_volume(3)


def test_cfg3_full_batch_u32_exact(mg, cfg3, vol3):
    g, c = cfg3
    boxes, extra = with_whole_volume(synth.make_boxes(3), c["dims"])
    h = run_plan(mg, g, torch.from_numpy(boxes).cuda(), "u32", c["name"])
    check_counts(h, boxes, c["dims"], Windows(3, vol3), c["S"], 24, 1 << 20, 5, vol_h=vol3, extra=extra)


def test_cfg3_fp16_weights_error_bound(mg, cfg3, vol3):
    g, c = cfg3
    boxes = synth.make_boxes(3, Q=20000)
    h = run_plan(mg, g, torch.from_numpy(boxes).cuda(), "f32", c["name"] + "-20k", alpha="f16")
    _, side = clipped(boxes, c["dims"])
    vol_q = side.prod(axis=1).astype(np.float64)
    assert np.allclose(h.astype(np.float64).sum(axis=1), vol_q, rtol=1e-5)
    D = g.info["depth"]
    win = Windows(3, vol3)
    idx = np.concatenate([sample_boxes(boxes, c["dims"], 16, 1 << 20, 6), largest_boxes(boxes, c["dims"], 4)])
    for i in idx:
        ref = win.hist(boxes[i, :3], side[i], c["S"]).astype(np.float64)
        # every pushed unit of weight crosses at most D rounded weights
        assert np.abs(h[i] - ref).sum() <= 1.5 * D * 2.0 ** -11 * vol_q[i] + 1e-3, i


def test_cfg3_propagate_f16_storage(mg, cfg3, vol3):
    g, c = cfg3
    tf = synth.make_tf(3, c["S"], 4)
    v32 = mg.mg_propagate_tf(g, torch.from_numpy(tf).cuda()).cpu().numpy()
    v16 = mg.mg_propagate_tf(g, torch.from_numpy(tf).cuda(), storage="f16").float().cpu().numpy()
    mg.mg_sync_status(g)
    D = g.info["depth"]
    win = Windows(3, vol3)

    def f16_check(x, ref, where):
        assert np.abs(np.asarray(x, np.float64) - ref).max() <= (2 * D + 1) * 2.0 ** -11, where

    voxel_colour_checks(mg, g, v32, win, tf, c["dims"], c["S"], (0, 2, 4, 6), 8, 7, fp32_check)
    voxel_colour_checks(mg, g, v16, win, tf, c["dims"], c["S"], (0, 2, 4, 6), 8, 7, f16_check)


# ---------------------------------------------------------------------------
# config 4: 614x961x600 cylinders, 15,917 segments; bf16 attribute TF frames
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg4(mg):
    c = synth.CONFIGS[4]
    vol_h = synth.make_volume(4)
    g = mg.mg_build(torch.from_numpy(vol_h).cuda(), c["S"])
    yield g, c, vol_h
    g.close()


def test_cfg4_full_batch_u32_exact(mg, cfg4):
    g, c, vol_h = cfg4
    boxes, extra = with_whole_volume(synth.make_boxes(4), c["dims"])
    h = run_plan(mg, g, torch.from_numpy(boxes).cuda(), "u32", c["name"])
    check_counts(h, boxes, c["dims"], Windows(4, vol_h), c["S"], 40, 1 << 23, 8, vol_h=vol_h, extra=extra)


def test_cfg4_bf16_attribute_frame(mg, cfg4):
    g, c, vol_h = cfg4
    tf = synth.make_attribute_tf(4, c["S"])
    samples = synth.make_samples(4)
    win = Windows(4, vol_h)
    D = g.info["depth"]
    for storage in ("f32", "bf16"):
        vals = mg.mg_propagate_tf(g, torch.from_numpy(tf).cuda(), storage=storage)
        look = mg.mg_render_lookup(g, vals, torch.from_numpy(samples).cuda()).float().cpu().numpy()
        mg.mg_sync_status(g)
        if storage == "f32":
            check = fp32_check
        else:
            def check(x, ref, where):
                assert np.abs(np.asarray(x, np.float64) - ref).max() <= (2 * D + 1) * 2.0 ** -8, where
        sample_colour_checks(mg, g, look, samples, c["dims"], win, tf, c["S"], 150, 9, check)
