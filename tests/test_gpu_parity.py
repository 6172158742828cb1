"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Integers (mip IDs, node table, node counts, depth, box histograms, cube
counts) must match bit for bit.  Floating point: |x - ref| <= 1e-5 |ref| or,
for |ref| < 1e-2, |x - ref| <= 1e-7, structural zeros exact (the stated FP32
tolerance); 16-bit storage is held to the bound its rounding allows.
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


def dev():
    return torch.device("cuda:0")


def build_pair(mg, vol, S, ids_dtype=None):
    t = torch.from_numpy(vol.astype(np.int32) if ids_dtype == "i32" else vol).to(dev())
    return mg.mg_build(t, S), oracle.Graph(vol, S)


VOLUMES = [
    ("cfg1-64^3", lambda: synth.make_volume(1), 64),
    ("ragged-37x29x23", lambda: synth.make_volume(1, dims=(37, 29, 23), S=24), 24),
    ("thin-130x7x3", lambda: synth.make_volume(1, dims=(130, 7, 3), S=50), 50),
    ("line-1x1x40", lambda: synth.make_volume(1, dims=(1, 1, 40), S=5), 5),
    ("one-voxel", lambda: np.array([[[2]]], np.uint16), 3),
    ("one-segment", lambda: np.zeros((17, 9, 12), np.uint16), 1),
    ("many-segments-40^3-s3000", lambda: synth.make_volume(1, dims=(40, 40, 40), S=3000), 3000),
    ("aniso-48x40x20", lambda: synth.make_volume(3, dims=(48, 40, 20), S=30), 30),
    ("powerlaw-45x33x27", lambda: synth.make_volume(2, dims=(45, 33, 27), S=40), 40),
]


@pytest.mark.parametrize("name,make,S", VOLUMES, ids=[v[0] for v in VOLUMES])
def test_build_bit_exact(mg, name, make, S):
    vol = make()
    g, og = build_pair(mg, vol, S)
    assert g.N == og.N and g.info["depth"] == og.D and g.info["levels"] == og.L
    assert g.info["bucket"] == og.bucket.tolist()
    assert g.info["max_list"] == og.max_nnz and g.info["pairs"] == og.pairs
    p, q, a, b = mg.mg_graph_copy_nodes(g)
    assert (p == og.p[: og.N]).all() and (q == og.q[: og.N]).all()
    assert (a == og.a[: og.N]).all() and (b == og.b[: og.N]).all()
    for level in range(og.L):
        assert (mg.mg_graph_copy_mip(g, level) == og.mip(level)).all(), level
    g.close()


def test_build_uint32_ids(mg):
    vol = synth.make_volume(1, dims=(33, 20, 17), S=70)
    g = mg.mg_build(torch.from_numpy(vol.astype(np.int32)).to(dev()), 70)
    og = oracle.Graph(vol, 70)
    assert g.N == og.N
    for level in range(og.L):
        assert (mg.mg_graph_copy_mip(g, level) == og.mip(level)).all()


def test_build_rejects_id_out_of_range(mg):
    vol = synth.make_volume(1, dims=(16, 16, 16), S=10)
    with pytest.raises(mg.MGError) as e:
        mg.mg_build(torch.from_numpy(vol).to(dev()), 9)
    assert e.value.status == mg.MG_ERR_INVALID_ARG


@pytest.mark.parametrize("C", [1, 3, 4, 16])
def test_propagate_fp32(mg, C):
    vol = synth.make_volume(1, dims=(37, 29, 23), S=24)
    g, og = build_pair(mg, vol, 24)
    tf = synth.make_tf(1, 24, C)
    vals = mg.mg_propagate_tf(g, torch.from_numpy(tf).to(dev())).cpu().numpy()
    ref = oracle.propagate(og.p, og.q, og.a, og.b, 24, tf.astype(np.float64))
    ok, err = fp32_close(vals, ref)
    assert ok, err
    # every voxel's colour is the direct convex combination (Sec. 3.4)
    for level in range(og.L):
        direct = oracle.direct_colors(vol, level, tf.astype(np.float64))
        ok, err = fp32_close(vals[og.mip(level).ravel()], direct)
        assert ok, (level, err)


@pytest.mark.parametrize("storage,u", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_propagate_16bit_storage_error_bound(mg, storage, u):
    vol = synth.make_volume(1)
    g, og = build_pair(mg, vol, 64)
    tf = synth.make_tf(1, 64, 4)
    vals = mg.mg_propagate_tf(g, torch.from_numpy(tf).to(dev()), storage=storage).float().cpu().numpy()
    ref = oracle.propagate(og.p, og.q, og.a, og.b, 64, tf.astype(np.float64))
    err = np.abs(vals - ref).max()
    # each level rounds the stored value (u) and the stored weight (u)
    bound = (2 * og.D + 1) * u
    assert err <= bound, (err, bound)


def _boxes_cfg1(Q=1000):
    return synth.make_boxes(1, Q=Q)


@pytest.mark.parametrize("schedule,chunk,threads", [("batched", 0, 0), ("batched", 64, 128), ("batched", 1000, 512),
                                                    ("plain", 0, 0)])
def test_query_u32_exact(mg, schedule, chunk, threads):
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 64)
    boxes = _boxes_cfg1(1000 if schedule == "batched" else 150)
    h = mg.mg_query_boxes(g, torch.from_numpy(boxes).to(dev()), schedule=schedule, chunk_cubes=chunk,
                          block_threads=threads).cpu().numpy()
    mg.mg_sync_status(g)
    ref = oracle.box_hist(vol, 64, boxes)
    assert np.array_equal(h, ref)


def test_query_csr_u32(mg):
    vol = synth.make_volume(1, dims=(37, 29, 23), S=24)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 24)
    boxes = synth.make_boxes(1, Q=300, dims=(37, 29, 23), box_max=40)
    off, seg, val = mg.mg_query_boxes(g, torch.from_numpy(boxes).to(dev()), layout="csr")
    off, seg, val = off.cpu().numpy(), seg.cpu().numpy(), val.cpu().numpy()
    ref = oracle.box_hist(vol, 24, boxes)
    for i in range(len(boxes)):
        nzs = np.nonzero(ref[i])[0]
        assert (seg[off[i]:off[i + 1]] == nzs).all()
        assert (val[off[i]:off[i + 1]] == ref[i][nzs]).all()
    # too small a capacity reports the size needed
    with pytest.raises(mg.MGError) as e:
        mg.mg_query_boxes(g, torch.from_numpy(boxes).to(dev()), layout="csr", capacity=3)
    assert e.value.status == mg.MG_ERR_CAPACITY


@pytest.mark.parametrize("layout", ["dense", "csr"])
def test_query_fp32(mg, layout):
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 64)
    boxes = _boxes_cfg1()
    ref = oracle.box_hist(vol, 64, boxes).astype(np.float64)
    if layout == "dense":
        h = mg.mg_query_boxes(g, torch.from_numpy(boxes).to(dev()), hist="f32").cpu().numpy()
    else:
        off, seg, val = [t.cpu().numpy() for t in mg.mg_query_boxes(g, torch.from_numpy(boxes).to(dev()),
                                                                     hist="f32", layout="csr")]
        h = np.zeros_like(ref)
        for i in range(len(boxes)):
            h[i, seg[off[i]:off[i + 1]]] = val[off[i]:off[i + 1]]
    ok, err = fp32_close(h, ref)
    assert ok, err


@pytest.mark.parametrize("alpha,u", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_query_16bit_weights_error_bound(mg, alpha, u):
    vol = synth.make_volume(1)
    g, og = build_pair(mg, vol, 64)
    boxes = _boxes_cfg1(400)
    ref = oracle.box_hist(vol, 64, boxes).astype(np.float64)
    h = mg.mg_query_boxes(g, torch.from_numpy(boxes).to(dev()), hist="f32", alpha=alpha).cpu().numpy()
    vol_q = np.prod(boxes[:, 3:].astype(np.float64), axis=1)
    l1 = np.abs(h - ref).sum(axis=1)
    # every pushed unit of weight crosses at most D rounded weights
    assert (l1 <= 1.5 * og.D * u * vol_q + 1e-3).all(), float((l1 / vol_q).max())
    assert np.allclose(h.sum(axis=1), vol_q, rtol=1e-5)


def test_count_cubes(mg):
    vol = synth.make_volume(1)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 64)
    boxes = _boxes_cfg1(500)
    c = mg.mg_count_cubes(g, torch.from_numpy(boxes).to(dev())).cpu().numpy()
    ref = np.array([oracle.fa_count(b, 64, 64, 64) for b in boxes], np.uint64)
    assert np.array_equal(c, ref)


def test_count_cubes_odd_dims_large_boxes(mg):
    # odd extents at every level and boxes up to the whole volume: many runs
    # per axis, both rising and falling, and clipping at the far faces
    rng = np.random.default_rng(77)
    dims = (300, 257, 129)
    vol = rng.integers(0, 8, size=dims[::-1], dtype=np.uint16)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 8)
    o = np.stack([rng.integers(0, d, 3000) for d in dims], 1)
    e = np.exp2(rng.uniform(0, 9.5, (3000, 3))).astype(np.int64)
    boxes = np.concatenate([o, e], 1).astype(np.int32)
    boxes[:5] = [[0, 0, 0, 300, 257, 129], [1, 1, 1, 299, 256, 128], [299, 256, 128, 1, 1, 1],
                 [3, 5, 7, 1000, 1000, 1000], [255, 127, 63, 2, 2, 2]]
    c = mg.mg_count_cubes(g, torch.from_numpy(boxes).to(dev())).cpu().numpy()
    ref = np.array([oracle.fa_count(b, *dims) for b in boxes], np.uint64)
    assert np.array_equal(c, ref)
    plan = mg.QueryPlan(g, max_Q=3000)
    h = plan.run(torch.from_numpy(boxes).to(dev())).cpu().numpy()
    mg.mg_sync_status(g)
    assert np.array_equal(h, oracle.box_hist(vol, 8, boxes))
    plan.close()


def test_query_edge_cases(mg):
    vol = synth.make_volume(1, dims=(19, 13, 11), S=12)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 12)
    boxes = np.array([[0, 0, 0, 19, 13, 11],      # whole volume
                      [18, 12, 10, 1, 1, 1],      # last voxel
                      [5, 3, 2, 100, 100, 100],   # clipped at the far faces
                      [0, 0, 0, 1, 1, 1],
                      [7, 0, 4, 1, 13, 1]], np.int32)
    h = mg.mg_query_boxes(g, torch.from_numpy(boxes).to(dev())).cpu().numpy()
    assert np.array_equal(h, oracle.box_hist(vol, 12, boxes))
    # empty batch
    e = mg.mg_query_boxes(g, torch.zeros((0, 6), dtype=torch.int32, device=dev()))
    assert e.shape == (0, 12)
    off, seg, val = mg.mg_query_boxes(g, torch.zeros((0, 6), dtype=torch.int32, device=dev()), layout="csr")
    assert off.cpu().numpy().tolist() == [0]
    # malformed boxes are reported through the status word, their rows stay zero
    bad = np.array([[0, 0, 0, 2, 2, 2], [19, 0, 0, 1, 1, 1], [0, 0, 0, 0, 1, 1], [-1, 0, 0, 1, 1, 1]], np.int32)
    h = mg.mg_query_boxes(g, torch.from_numpy(bad).to(dev())).cpu().numpy()
    with pytest.raises(mg.MGError) as ei:
        mg.mg_sync_status(g)
    assert ei.value.status == mg.MG_ERR_INVALID_ARG
    assert np.array_equal(h[0], oracle.box_hist(vol, 12, bad[:1])[0])
    assert (h[1:] == 0).all()
    mg.mg_sync_status(g)   # cleared


def test_render_lookup(mg):
    dims = (37, 29, 23)
    vol = synth.make_volume(1, dims=dims, S=24)
    g, og = build_pair(mg, vol, 24)
    tf = synth.make_tf(1, 24, 4)
    vals_t = mg.mg_propagate_tf(g, torch.from_numpy(tf).to(dev()))
    smp = synth.make_samples(1, dims=dims, width=160, height=90)
    smp[:7] = [[0, 0, 0, 0], [-3, 40, 1e9, 2.49], [np.nan, 5, 5, np.nan], [36.99, 28.99, 22.99, -1],
               [18.5, 14.5, 11.5, 100], [36.5, 28.5, 22.5, 1.5], [1e-8, 1e-8, 1e-8, 0.5]]
    out = mg.mg_render_lookup(g, vals_t, torch.from_numpy(smp).to(dev())).cpu().numpy()
    vals = vals_t.cpu().numpy()
    lev, vox = oracle.sample_voxels(og.dims, smp)
    nodes = np.array([og.mip(int(l)).ravel()[v] for l, v in zip(lev, vox)])
    assert np.array_equal(out, vals[nodes])
    # and the colour is the direct convex combination of that voxel
    direct = {l: oracle.direct_colors(vol, l, tf.astype(np.float64)) for l in set(lev.tolist())}
    ref = np.stack([direct[int(l)][v] for l, v in zip(lev, vox)])
    ok, err = fp32_close(out, ref)
    assert ok, err
    # bf16 values are copied bit for bit
    vb = mg.mg_propagate_tf(g, torch.from_numpy(tf).to(dev()), storage="bf16")
    ob = mg.mg_render_lookup(g, vb, torch.from_numpy(smp).to(dev()))
    assert torch.equal(ob.cpu(), vb.cpu()[torch.from_numpy(nodes.astype(np.int64))])


@pytest.mark.parametrize("cfg,dims,S", [(1, (64, 64, 64), 64), (2, (45, 33, 27), 40), (3, (48, 40, 20), 30)])
def test_generators_agree(cfg, dims, S):
    """The GPU volume generator reproduces the host generator bit for bit."""
    host = synth.make_volume(cfg, dims=dims, S=S)
    gpu = synth.make_volume(cfg, device="cuda", dims=dims, S=S).cpu().numpy()
    assert np.array_equal(host, gpu)


@pytest.mark.parametrize("k,C,storage", [(3, 4, "f32"), (8, 4, "f32"), (5, 4, "f16"), (2, 16, "bf16"), (7, 3, "f32")])
def test_propagate_multi_tf(mg, k, C, storage):
    """k TFs in one pass: slice j of every row equals the single-TF propagation
    of TF j bit for bit, and (fp32) the oracle's fp64 lerps within tolerance."""
    vol = synth.make_volume(1, dims=(37, 29, 23), S=24)
    g, og = build_pair(mg, vol, 24)
    tfs = np.stack([synth.make_tf(1, 24, C, frame=j) for j in range(k)])
    if k * C not in (1, 2, 3, 4, 5, 6, 7, 8, 12, 16, 20, 24, 28, 32):
        with pytest.raises(mg.MGError) as e:
            mg.mg_propagate_tf_multi(g, torch.from_numpy(tfs).to(dev()), storage=storage)
        assert e.value.status == mg.MG_ERR_UNSUPPORTED
        return
    vals = mg.mg_propagate_tf_multi(g, torch.from_numpy(tfs).to(dev()), storage=storage)
    mg.mg_sync_status(g)
    for j in range(k):
        one = mg.mg_propagate_tf(g, torch.from_numpy(tfs[j]).to(dev()), storage=storage)
        assert torch.equal(vals[:, j * C:(j + 1) * C].cpu(), one.cpu()), j
        if storage == "f32":
            ref = oracle.propagate(og.p, og.q, og.a, og.b, 24, tfs[j].astype(np.float64))
            ok, err = fp32_close(vals[:, j * C:(j + 1) * C].cpu().numpy(), ref)
            assert ok, (j, err)


def test_render_lookup_multi(mg):
    dims = (37, 29, 23)
    vol = synth.make_volume(1, dims=dims, S=24)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 24)
    k, C = 4, 4
    tfs = np.stack([synth.make_tf(1, 24, C, frame=j) for j in range(k)])
    for storage in ("f32", "f16"):
        vals = mg.mg_propagate_tf_multi(g, torch.from_numpy(tfs).to(dev()), storage=storage)
        frames = [synth.make_samples(1, dims=dims, width=w, height=h, frame=j)
                  for j, (w, h) in enumerate([(40, 30), (1, 1), (2, 1), (64, 17)])]
        frames[2] = frames[2][:0]   # a frame without samples
        off = np.cumsum([0] + [len(f) for f in frames])
        smp = torch.from_numpy(np.concatenate(frames)).to(dev())
        out = mg.mg_render_lookup_multi(g, vals, k, smp, off).cpu()
        for j in range(k):
            if off[j + 1] == off[j]:
                continue
            one = mg.mg_render_lookup(g, vals[:, j * C:(j + 1) * C].contiguous(),
                                      torch.from_numpy(frames[j]).to(dev())).cpu()
            assert torch.equal(out[off[j]:off[j + 1]], one), (storage, j)
    g.close()


# the ray marcher (Sec. 4): decisions in fp32 as the oracle takes them, so the
# samples per pixel match exactly; colours differ only through the node values
# (fp32 lerps here, fp64 lerps rounded to fp32 in the oracle) and log2 of the
# level fraction: a few fp32 ulps per sample over at most a few hundred samples
MARCH_TOL = 2e-5
MARCH_CASES = [
    ("voronoi-lod4", 1, (48, 40, 36), 30, dict(lod_bias=4, ert=2.0, base_step=0.5)),
    ("voronoi-lod0-ert", 2, (45, 33, 27), 40, dict(lod_bias=0, ert=0.95, base_step=0.25)),
    ("cylinders-lod0", 4, (64, 64, 64), 4, dict(lod_bias=0, ert=2.0, base_step=0.5)),
    ("cylinders-lod-2", 4, (64, 64, 64), 12, dict(lod_bias=-2, ert=0.99, base_step=0.5)),
]


@pytest.mark.parametrize("name,cfg,dims,S,kw", MARCH_CASES, ids=[c[0] for c in MARCH_CASES])
def test_raymarch_matches_oracle(mg, name, cfg, dims, S, kw):
    vol = synth.make_volume(cfg, dims=dims, S=S)
    g, og = build_pair(mg, vol, S)
    tf = synth.make_attribute_tf(cfg, S) if cfg == 4 else synth.make_tf(cfg, S, 4)
    vals = mg.mg_propagate_tf(g, torch.from_numpy(tf).to(dev()))
    ref_vals = oracle.propagate(og.p, og.q, og.a, og.b, S, tf.astype(np.float64)).astype(np.float32)
    cam = synth.orbit_camera(cfg, dims=dims, width=96, height=64, **kw)
    img, steps = mg.mg_raymarch(g, vals, cam, steps=True)
    opac = vals[:, 3].contiguous()
    img_ess, steps_ess = mg.mg_raymarch(g, vals, cam, opacity=opac, steps=True)
    mg.mg_sync_status(g)
    # skipping passes over samples of zero opacity only: the same image
    assert torch.equal(img.cpu(), img_ess.cpu())
    assert bool((steps_ess <= steps).all())
    ref, ref_steps, margin = og.raymarch(ref_vals, cam)
    ref_e, ref_steps_e, _ = og.raymarch(ref_vals, cam, opacity=ref_vals[:, 3].copy())
    # pixels whose early termination was decided within 1e-4 of the threshold
    # may stop one sample apart; every other pixel takes the same samples
    ok = margin >= 1e-4
    assert ok.mean() > 0.95
    got, got_steps = img.cpu().numpy(), steps.cpu().numpy()
    assert np.array_equal(got_steps[ok], ref_steps[ok])
    assert np.array_equal(steps_ess.cpu().numpy()[ok], ref_steps_e[ok])
    assert np.abs(got[ok] - ref[ok]).max() <= MARCH_TOL
    assert (got[..., 3] <= 1.0 + 1e-6).all() and (got >= 0).all()
    g.close()


def test_raymarch_argument_checks(mg):
    vol = synth.make_volume(1, dims=(16, 16, 16), S=8)
    g = mg.mg_build(torch.from_numpy(vol).to(dev()), 8)
    vals = mg.mg_propagate_tf(g, torch.from_numpy(synth.make_tf(1, 8, 4)).to(dev()))
    cam = synth.orbit_camera(1, dims=(16, 16, 16), width=8, height=8)
    for bad in (dict(width=0), dict(pix=0.0), dict(base_step=-1.0), dict(max_steps=0), dict(lod_bias=100)):
        with pytest.raises(mg.MGError) as e:
            mg.mg_raymarch(g, vals, dict(cam, **bad))
        assert e.value.status == mg.MG_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        mg.mg_raymarch(g, vals[:, :3], cam)
    g.close()


# the bitstream (Table 1): encoded on the GPU byte for byte as the oracle
# writes it, decoded on the GPU back to the graph, looked up in place
@pytest.mark.parametrize("dims,S", [((37, 29, 23), 24), ((64, 64, 64), 64), ((16, 16, 16), 1), ((130, 7, 3), 50)])
def test_bitstream_matches_oracle_and_decodes(mg, dims, S):
    vol = synth.make_volume(1, dims=dims, S=S) if S > 1 else np.zeros(dims[::-1], np.uint16)
    g, og = build_pair(mg, vol, S)
    bs = mg.mg_bitstream_write(g)
    ref = og.bitstream()
    assert bs.data.cpu().numpy().tobytes() == ref
    assert bs.info.bytes == len(ref) and bs.info.num_nodes == og.N
    for level in range(og.L):
        assert np.array_equal(bs.decode_mip(level).cpu().numpy(), og.mip(level)), level
    p, q, a, b = (t.cpu().numpy() for t in bs.decode_nodes())
    assert (p == og.p[:og.N]).all() and (q == og.q[:og.N]).all()
    assert (a == og.a[:og.N]).all() and (b == og.b[:og.N]).all()
    tf = torch.from_numpy(synth.make_tf(1, S, 4)).to(dev())
    for storage in ("f32", "bf16"):
        vals = mg.mg_propagate_tf(g, tf, storage=storage)
        smp = torch.from_numpy(synth.make_samples(1, dims=dims, width=64, height=40)).to(dev())
        assert torch.equal(bs.lookup(vals, smp).cpu(), mg.mg_render_lookup(g, vals, smp).cpu())
    g.close()


# greedy factorisation (Sec. 3.3, Sec. 3.7): integer decisions throughout, so
# the GPU graph equals the oracle's bit for bit; sigma is an fp64 sum
@pytest.mark.parametrize("strategy,tau,bitrate,cfg,dims,S", [
    ("reduction", 3, 9, 1, (24, 20, 16), 20),
    ("occurrence", 3, 9, 1, (24, 20, 16), 20),
    ("reduction", 3, 0, 2, (21, 14, 11), 15),
    ("reduction", 1, 5, 3, (33, 17, 9), 12),
    ("occurrence", 2, 16, 1, (32, 32, 32), 24),
])
def test_greedy_matches_oracle(mg, strategy, tau, bitrate, cfg, dims, S):
    vol = synth.make_volume(cfg, dims=dims, S=S)
    r = mg.mg_factor_greedy(torch.from_numpy(vol).to(dev()), S, strategy=strategy, tau=tau, bitrate=bitrate)
    og, cb, sg, picks = oracle.greedy(vol, S, strategy, tau=tau, bitrate=bitrate)
    assert r["N"] == og.N and r["D"] == og.D and r["L"] == og.L
    assert np.array_equal(r["picks"], picks)
    for k in "pqab":
        assert np.array_equal(r[k], getattr(og, k)[:og.N]), k
    for l in range(og.L):
        assert np.array_equal(r["mip"][l], og.mip(l)), l
    if bitrate:
        assert np.array_equal(r["codebook"], cb)
        assert np.allclose(r["sigma"], sg, rtol=1e-9, atol=1e-15)


# mixture table with uncertainties (Sec. 3.5) and the table-summed query
def _rows_close(got, ref):
    off, src, mu, dmu = got
    roff, rsrc, rmu, rdmu = ref
    assert np.array_equal(off, roff) and np.array_equal(src, rsrc)
    assert np.allclose(mu, rmu, rtol=1e-12, atol=1e-15) and np.allclose(dmu, rdmu, rtol=1e-9, atol=1e-15)


def test_error_table_and_lut_query_exact_graph(mg):
    dims, S = (37, 29, 23), 24
    vol = synth.make_volume(1, dims=dims, S=S)
    g, og = build_pair(mg, vol, S)
    _rows_close(mg.mg_error_table(g), oracle.error_rows(og, *oracle.node_weights(og)))
    boxes = synth.make_boxes(1, Q=300, dims=dims, box_max=40)
    h, e = mg.mg_query_lut(g, torch.from_numpy(boxes).to(dev()))
    mg.mg_sync_status(g)
    assert np.allclose(h.cpu().numpy(), oracle.box_hist(vol, S, boxes), rtol=1e-12, atol=1e-9)
    assert (e.cpu().numpy() == 0).all()
    g.close()


@pytest.mark.parametrize("bitrate", [4, 9])
def test_quantised_graph_table_queries_and_colours(mg, bitrate):
    dims, S = (24, 20, 16), 20
    vol = synth.make_volume(1, dims=dims, S=S)
    r = mg.mg_factor_greedy(torch.from_numpy(vol).to(dev()), S, "reduction", tau=3, bitrate=bitrate, graph=True)
    g = r["graph"]
    og, cb, sg, _ = oracle.greedy(vol, S, "reduction", tau=3, bitrate=bitrate)
    rows = oracle.error_rows(og, *oracle.node_weights(og, cb, sg))
    _rows_close(mg.mg_error_table(g), rows)
    boxes = synth.make_boxes(1, Q=200, dims=dims, box_max=24)
    bt = torch.from_numpy(boxes).to(dev())
    h, e = mg.mg_query_lut(g, bt)
    hr, er = oracle.lut_query(og, rows, boxes)
    assert np.allclose(h.cpu().numpy(), hr, rtol=1e-10, atol=1e-9)
    assert np.allclose(e.cpu().numpy(), er, rtol=1e-9, atol=1e-12) and (er > 0).any()
    # the fp32 push through the codeword weights gives the same expectations
    hf = mg.mg_query_boxes(g, bt, hist="f32").cpu().numpy()
    assert np.allclose(hf, hr, rtol=1e-4, atol=1e-2)
    with pytest.raises(mg.MGError) as ex:
        mg.mg_query_boxes(g, bt)
    assert ex.value.status == mg.MG_ERR_UNSUPPORTED
    # colours: the codeword lerps of Sec. 3.4 = sum over a node's row of mu * TF
    tf = synth.make_tf(1, S, 4)
    vals = mg.mg_propagate_tf(g, torch.from_numpy(tf).to(dev())).cpu().numpy()
    off, src, mu, _ = rows
    ref = np.stack([mu[off[n]:off[n + 1]] @ tf[src[off[n]:off[n + 1]]].astype(np.float64) for n in range(og.N)])
    ok, err_ = fp32_close(vals, ref)
    assert ok, err_
    mg.mg_sync_status(g)
    g.close()
