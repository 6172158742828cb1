"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each expected value is printed
in the paper (tests/golden/*.json, cited there), worked by hand from the
paper's definitions, a closed form, an invariant, or a brute-force count by a
different code path.
"""
from fractions import Fraction
from math import gcd

import numpy as np
import pytest

import oracle
from paper_2009_02702_gb300 import synth
from tests.conftest import golden


def F(s):
    return Fraction(s)


# --------------------------------------------------------------------------
# Eq. 4 / Table 2: mip geometry
# --------------------------------------------------------------------------
def test_table2_voxel_totals_and_levels():
    g = golden("table2_mip_geometry.json")
    for ds in g["datasets"]:
        dims = oracle.level_dims(*ds["resolution"])
        assert dims.shape[0] == ds["mip_levels"], ds["name"]
        total = int(np.prod(dims, axis=1).sum())
        printed = ds["voxels_million"].replace(",", "")
        decimals = len(printed.split(".")[1]) if "." in printed else 0
        # the paper truncates (1,195,445,766 -> 1,195) or rounds to its digits
        assert abs(total / 1e6 - float(printed)) < 10 ** -decimals, (ds["name"], total)
        assert tuple(dims[-1]) == (1, 1, 1)


def test_level_dims_round_up():
    d = oracle.level_dims(5, 1, 3)
    assert d.tolist() == [[5, 1, 3], [3, 1, 2], [2, 1, 1], [1, 1, 1]]
    assert oracle.level_dims(1, 1, 1).tolist() == [[1, 1, 1]]


# --------------------------------------------------------------------------
# Eq. 4: mixtures, hand-worked border cases and invariants
# --------------------------------------------------------------------------
def _vol_from_case(case):
    nx, ny, nz = case["dims"]
    if "ids" in case:
        return np.array(case["ids"], np.uint16).reshape(nz, ny, nx)
    v = np.zeros((nz, ny, nx), np.uint16)
    x, y, z = case["ids_corner_one"]
    v[z, y, x] = 1
    return v


def test_eq4_hand_worked_border_cases():
    g = golden("eq4_border_mixtures.json")
    for case in g["cases"]:
        vol = _vol_from_case(case)
        for lev, voxels in case["levels"].items():
            off, ids, cnt = oracle.mixtures(vol, int(lev))
            assert off.shape[0] - 1 == len(voxels)
            for v, entries in enumerate(voxels):
                got = [[int(i), int(c)] for i, c in zip(ids[off[v]:off[v + 1]], cnt[off[v]:off[v + 1]])]
                assert got == entries, (case["dims"], lev, v)
        if "level1_corner_voxel" in case:
            off, ids, cnt = oracle.mixtures(vol, 1)
            v = 7  # (1,1,1) in a 2x2x2 level
            got = [[int(i), int(c)] for i, c in zip(ids[off[v]:off[v + 1]], cnt[off[v]:off[v + 1]])]
            assert got == case["level1_corner_voxel"]


def test_eq1_eq2_invariants_and_interior_counts():
    vol = synth.make_volume(1, dims=(24, 20, 18), S=16)
    dims = oracle.level_dims(24, 20, 18)
    for l in range(dims.shape[0]):
        off, ids, cnt = oracle.mixtures(vol, l)
        nx, ny, nz = dims[l]
        assert off.shape[0] - 1 == nx * ny * nz
        for v in range(nx * ny * nz):
            e = slice(off[v], off[v + 1])
            assert off[v + 1] > off[v]
            assert int(cnt[e].sum()) == 8 ** l                       # Eq. 1 (x 8^l)
            assert (cnt[e] >= 1).all()                                # Eq. 2
            assert (np.diff(ids[e].astype(np.int64)) > 0).all()       # sorted, unique
        # interior voxels (whole 2^l footprint inside): raw counts of level-0 IDs
        s = 2 ** l
        for Z in range(nz):
            for Y in range(ny):
                for X in range(nx):
                    if (X + 1) * s > 24 or (Y + 1) * s > 20 or (Z + 1) * s > 18:
                        continue
                    sub = vol[Z * s:(Z + 1) * s, Y * s:(Y + 1) * s, X * s:(X + 1) * s].ravel()
                    bc = np.bincount(sub, minlength=16)
                    v = (Z * ny + Y) * nx + X
                    e = slice(off[v], off[v + 1])
                    dense = np.zeros(16, np.int64)
                    dense[ids[e]] = cnt[e]
                    assert (dense == bc).all()


def test_level0_is_lossless():
    vol = synth.make_volume(1, dims=(9, 7, 5), S=10)
    off, ids, cnt = oracle.mixtures(vol, 0)
    assert (np.diff(off) == 1).all() and (cnt == 1).all()
    assert (ids == vol.ravel()).all()
    g = oracle.Graph(vol, 10)
    assert (g.mip(0) == vol).all()


# --------------------------------------------------------------------------
# Sec. 3.2-3.3: factorisation, Fig. 2 / Fig. 3 / Fig. 4
# --------------------------------------------------------------------------
def _paper_table_fig3():
    """The Fig. 2/3 tree as an oracle node table (sources 0..3 = e1..e4)."""
    g = golden("fig2_fig3_factorization.json")
    name_to_id = {str(i + 1): i for i in range(4)}
    p, q, a, b = [oracle.NONE] * 4, [oracle.NONE] * 4, [0] * 4, [0] * 4
    for name in ("5", "6", "7"):
        nd = g["nodes"][name]
        wi, wj = F(nd["edge_weight"][0]), F(nd["edge_weight"][1])
        assert wi + wj == 1
        den = wi.denominator * wj.denominator // gcd(wi.denominator, wj.denominator)
        name_to_id[name] = len(p)
        p.append(name_to_id[str(nd["pred"][0])])
        q.append(name_to_id[str(nd["pred"][1])])
        a.append(int(wi * den))
        b.append(int(wj * den))
    return g, name_to_id, np.array(p), np.array(q), np.array(a), np.array(b)


def test_fig2_fig3_expansion():
    g, ids, p, q, a, b = _paper_table_fig3()
    for name, expect in g["expanded"].items():
        fr = [F(x) for x in expect]
        den = 1
        for x in fr:
            den = den * x.denominator // gcd(den, x.denominator)
        out = oracle.expand(p, q, a, b, 4, ids[name], den)
        assert [Fraction(int(v), den) for v in out] == fr, name
    # Sec. 3.4: levels of the chain
    assert oracle.depths(p, q, 4).tolist() == [0, 0, 0, 0, 1, 2, 3]


def test_fig2_propagation_of_unit_vectors():
    g, ids, p, q, a, b = _paper_table_fig3()
    val = oracle.propagate(p, q, a, b, 4, np.eye(4))
    m = [float(F(x)) for x in g["mixture"]]
    assert np.allclose(val[ids["7"]], m, rtol=0, atol=1e-15)


def test_fig4_reuse_of_lambda5():
    g = golden("fig4_dag.json")
    lists = []
    for mix in g["mixtures"]:
        fr = [F(x) for x in mix]
        lists.append([(i, int(x * 10)) for i, x in enumerate(fr)])
    G, roots = oracle.factor_lists(lists, 4)
    # exactly one node mixes e1 and e2 at 1:2 and both mixtures use it
    sh = g["shared_node"]
    wi, wj = F(sh["edge_weight"][0]), F(sh["edge_weight"][1])
    key = (sh["pred"][0] - 1, sh["pred"][1] - 1, int(wi * 3), int(wj * 3))
    hits = [k for k in range(G.N) if (G.p[k], G.q[k], G.a[k], G.b[k]) == key]
    assert len(hits) == 1
    lam5 = hits[0]
    # m' = 3/5 lambda_5 + 2/5 lambda_8, lambda_8 = 1/4 e3 + 3/4 e4
    r1 = int(roots[1])
    assert G.p[r1] == lam5 and (G.a[r1], G.b[r1]) == (3, 2)
    l8 = int(G.q[r1])
    assert (G.p[l8], G.q[l8], G.a[l8], G.b[l8]) == (2, 3, 1, 3)
    # m reaches lambda_5 through its root's left subtree
    r0 = int(roots[0])
    assert G.p[r0] == lam5
    for r, lst in zip(roots, lists):
        out = oracle.expand(G.p, G.q, G.a, G.b, 4, int(r), 10)
        assert out.tolist() == [w for _, w in lst]


def test_fig5_topological_levels():
    g = golden("fig5_topological_levels.json")
    names = g["node_names"]
    idx = {n: i for i, n in enumerate(names)}
    S = g["sources"]
    p = np.full(len(names), oracle.NONE, np.uint32)
    q = np.full(len(names), oracle.NONE, np.uint32)
    for n, (u, v) in g["edges_into"].items():
        p[idx[n]], q[idx[n]] = idx[u], idx[v]
    lev = oracle.depths(p, q, S)
    assert lev.tolist() == g["levels"]
    # the deferrable node: its successors' minimum level bounds its window
    node = idx[g["deferrable"]["node"]]
    succ_levels = [lev[idx[n]] for n, pr in g["edges_into"].items() if names[node] in pr]
    assert list(range(lev[node], min(succ_levels))) == g["deferrable"]["may_run_with_levels"]


# --------------------------------------------------------------------------
# Sec. 3.2-3.4 on whole volumes: pruning keeps every mixture, table structure
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims,S", [((16, 16, 16), 8), ((13, 9, 11), 12), ((1, 1, 40), 5)])
def test_graph_expansion_equals_mixtures(dims, S):
    vol = synth.make_volume(1, dims=dims, S=S)
    g = oracle.Graph(vol, S)
    for l in range(g.L):
        off, ids, cnt = oracle.mixtures(vol, l)
        mip = g.mip(l).ravel()
        for v in range(mip.shape[0]):
            out = oracle.expand(g.p, g.q, g.a, g.b, S, int(mip[v]), 8 ** l)
            dense = np.zeros(S, np.uint64)
            dense[ids[off[v]:off[v + 1]]] = cnt[off[v]:off[v + 1]]
            assert (out == dense).all(), (l, v)


def test_graph_table_structure():
    vol = synth.make_volume(1, dims=(32, 24, 20), S=20)
    g = oracle.Graph(vol, 20)
    S = g.S
    k = np.arange(S, g.N)
    # Eq. 8: predecessors come first
    assert (g.p[S:] < k).all() and (g.q[S:] < k).all()
    # reduced ratios
    assert (g.a[S:] >= 1).all() and (g.b[S:] >= 1).all()
    assert all(gcd(int(x), int(y)) == 1 for x, y in zip(g.a[S:], g.b[S:]))
    # Sec. 3.4 levels and buckets
    assert (g.depth == oracle.depths(g.p, g.q, S)).all()
    assert g.bucket[0] == 0 and g.bucket[1] == S and g.bucket[-1] == g.N
    for d in range(1, g.D + 1):
        assert (g.depth[g.bucket[d]:g.bucket[d + 1]] == d).all()
    # canonical order inside each bucket, and unique keys (pruning)
    keys = list(zip(g.depth[S:], g.p[S:], g.q[S:], g.a[S:], g.b[S:]))
    assert keys == sorted(keys)
    assert len(set(keys)) == len(keys)


def test_two_segment_node_count_is_distinct_ratios():
    """With two segments every mixed voxel is one lerp of the two sources, so
    the number of internal nodes is the number of distinct reduced ratios."""
    vol = np.zeros((20, 20, 20), np.uint16)
    zz, yy, xx = np.meshgrid(np.arange(20), np.arange(20), np.arange(20), indexing="ij")
    vol[(3 * xx + 5 * yy + 7 * zz) > 150] = 1
    g = oracle.Graph(vol, 2)
    ratios = set()
    for l in range(1, g.L):
        off, ids, cnt = oracle.mixtures(vol, l)
        for v in range(off.shape[0] - 1):
            if off[v + 1] - off[v] == 2:
                c0, c1 = int(cnt[off[v]]), int(cnt[off[v] + 1])
                t = gcd(c0, c1)
                ratios.add((c0 // t, c1 // t))
    assert g.N - 2 == len(ratios)
    assert g.D == 1


# --------------------------------------------------------------------------
# Sec. 3.4 / Sec. 4: forward propagation equals the direct convex combination
# --------------------------------------------------------------------------
def test_propagation_equals_direct_sum():
    vol = synth.make_volume(1, dims=(20, 18, 16), S=30)
    g = oracle.Graph(vol, 30)
    tf = synth.make_tf(1, 30, 4).astype(np.float64)
    val = oracle.propagate(g.p, g.q, g.a, g.b, 30, tf)
    for l in range(g.L):
        direct = oracle.direct_colors(vol, l, tf)
        got = val[g.mip(l).ravel()]
        assert np.allclose(got, direct, rtol=1e-12, atol=1e-14)


def test_unit_vector_tf_gives_mixtures():
    vol = synth.make_volume(1, dims=(12, 12, 12), S=9)
    g = oracle.Graph(vol, 9)
    val = oracle.propagate(g.p, g.q, g.a, g.b, 9, np.eye(9))
    for l in range(g.L):
        off, ids, cnt = oracle.mixtures(vol, l)
        mip = g.mip(l).ravel()
        for v in range(mip.shape[0]):
            dense = np.zeros(9)
            dense[ids[off[v]:off[v + 1]]] = cnt[off[v]:off[v + 1]] / 8.0 ** l
            assert np.allclose(val[mip[v]], dense, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------
# Sec. 3.6: brute-force histograms, footprint assembly
# --------------------------------------------------------------------------
def test_box_hist_brute_force_and_clipping():
    vol = synth.make_volume(1, dims=(17, 13, 11), S=7)
    rng = np.random.default_rng(5)
    boxes = []
    for _ in range(200):
        o = [rng.integers(0, n) for n in (17, 13, 11)]
        s = [rng.integers(1, 2 * n) for n in (17, 13, 11)]   # often past the border
        boxes.append(o + s)
    boxes = np.array(boxes, np.int32)
    h = oracle.box_hist(vol, 7, boxes)
    for bx, row in zip(boxes, h):
        x, y, z, dx, dy, dz = bx
        sub = vol[z:z + dz, y:y + dy, x:x + dx]
        assert (np.bincount(sub.ravel(), minlength=7) == row).all()
        assert row.sum() == sub.size


def test_fig6_footprint_example():
    g = golden("fig6_footprint.json")
    assert oracle.footprint_1d(g["x_range"][0], g["x_range"][1], 1 << 20) == g["x_levels"]
    assert oracle.footprint_1d(g["y_range"][0], g["y_range"][1], 1 << 20) == g["y_levels"]
    box = [g["x_range"][0], g["y_range"][0], 0, g["x_range"][1], g["y_range"][1], 4]
    cubes = oracle.fa_cubes(box, 64, 64, 64)
    per = {int(l): int(c) for l, c in zip(*np.unique(cubes[:, 0], return_counts=True))}
    sq = {int(k): v for k, v in g["squares_per_level"].items()}
    assert per == {l: n * 2 ** (2 - l) for l, n in sq.items()}


def test_footprint_1d_hand_cases():
    assert oracle.footprint_1d(0, 16, 100) == [4]
    assert oracle.footprint_1d(1, 512, 4096) == [0, 1, 2, 3, 4, 5, 6, 7, 8, 0]
    assert oracle.footprint_1d(5, 100, 8) == [0, 1]            # clipped to [5, 8)
    assert oracle.footprint_1d(0, 7, 7) == [2, 1, 0]
    assert oracle.footprint_1d(6, 1, 7) == [0]


def test_fa_cubes_tile_the_clipped_box():
    dims = (23, 17, 14)
    rng = np.random.default_rng(11)
    for _ in range(150):
        o = [int(rng.integers(0, n)) for n in dims]
        s = [int(rng.integers(1, n + 6)) for n in dims]
        box = o + s
        cubes = oracle.fa_cubes(box, *dims)
        mark = np.zeros(dims[::-1], np.int32)
        for l, x, y, z in cubes:
            e = 1 << l
            assert x * e >= o[0] and y * e >= o[1] and z * e >= o[2]
            mark[z * e:(z + 1) * e, y * e:(y + 1) * e, x * e:(x + 1) * e] += 1
        want = np.zeros_like(mark)
        want[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]] = 1
        assert (mark == want).all(), box


def test_fa_cube_count_closed_form():
    # Algorithm 1's block of run levels (a, b, c) holds 2^(a+b+c-3m) cubes at
    # level m = min(a, b, c).  With F(m) = sum over an axis's steps of level
    # >= m of 2^(level-m) and P(m) = Fx Fy Fz, every block adds 2^(a+b+c-3m')
    # to P(m') for each m' <= m, so the total is P(0) - 7 * sum_{m>=1} P(m):
    # a count that never lists the blocks.
    rng = np.random.default_rng(23)
    for _ in range(400):
        dims = [int(rng.choice([7, 64, 300, 384, 961, 2048])) for _ in range(3)]
        o = [int(rng.integers(0, n)) for n in dims]
        s = [int(2 ** rng.uniform(0, 11.5)) for _ in range(3)]
        steps = [oracle.footprint_1d(o[k], s[k], dims[k]) for k in range(3)]

        def F(levels, m):
            return sum(1 << (lv - m) for lv in levels if lv >= m)

        P = [F(steps[0], m) * F(steps[1], m) * F(steps[2], m) for m in range(40)]
        closed = P[0] - 7 * sum(P[1:])
        assert oracle.fa_count(o + s, *dims) == closed, (dims, o, s)
        assert P[0] == np.prod([min(o[k] + s[k], dims[k]) - o[k] for k in range(3)])


def test_fa_query_equals_brute_force():
    vol = synth.make_volume(1)
    g = oracle.Graph(vol, 64)
    boxes = synth.make_boxes(1, Q=300)
    assert (g.fa_query(boxes) == oracle.box_hist(vol, 64, boxes)).all()


def test_table3_saved_arithmetic():
    g = golden("table3_fetches.json")
    for ds, fetches in g["fetches"].items():
        for size, f, saved in zip(g["sizes"], fetches, g["saved_percent"][ds]):
            mult = 1000.0 if f.endswith("K") else 1.0
            digits = f.rstrip("K")
            dec = len(digits.split(".")[1]) if "." in digits else 0
            half = 0.5 * 10 ** -dec * mult
            lo = 100 * (1 - (float(digits) * mult + half) / size ** 3)
            hi = 100 * (1 - (float(digits) * mult - half) / size ** 3)
            s = float(saved)
            assert lo - 0.006 <= s <= hi + 0.006, (ds, size)


def test_table3_fetch_counts_sanity_band():
    """Randomly aligned cubic regions: mean fetch count within +-25% of the
    paper's range (the paper's sampling is not specified: a band, not a pin)."""
    g = golden("table3_fetches.json")
    rng = np.random.default_rng(3)
    big = 4096
    for si, size in enumerate(g["sizes"]):
        vals = []
        for ds in g["fetches"].values():
            f = ds[si]
            vals.append(float(f.rstrip("K")) * (1000.0 if f.endswith("K") else 1.0))
        n = 400 if size <= 64 else 60
        counts = [oracle.fa_count([int(rng.integers(0, big - size)) for _ in range(3)] + [size] * 3,
                                  big, big, big) for _ in range(n)]
        m = float(np.mean(counts))
        assert 0.75 * min(vals) <= m <= 1.25 * max(vals), (size, m, vals)


def test_sec4_sample_lookup_hand_cases():
    g = golden("sec4_sample_lookup.json")
    dims = oracle.level_dims(*g["dims"])
    smp = np.array([[float(x) for x in s["xyzl"]] for s in g["samples"]], np.float32)
    lev, vox = oracle.sample_voxels(dims, smp)
    for s, l, v in zip(g["samples"], lev, vox):
        assert l == s["level"]
        nx, ny, _ = dims[l]
        x, y, z = s["voxel"]
        assert v == (z * ny + y) * nx + x, s


# ---------------------------------------------------------------------------
# Sec. 4: the ray marcher
# ---------------------------------------------------------------------------
def _march_cam(eye, width=24, height=16, base=0.5, bias=-64, ert=2.0, max_steps=1 << 20, target=None):
    eye = np.array(eye, np.float64)
    target = np.array(target if target is not None else eye + [1.0, 0.3, 0.2], np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    f32 = lambda v: [float(np.float32(x)) for x in v]
    return dict(eye=f32(eye), fwd=f32(fwd), right=f32(right), up=f32(up), pix=float(np.float32(0.01)),
                width=width, height=height, base_step=base, lod_bias=bias, ert=ert, max_steps=max_steps)


def _ray_dirs(cam):
    """fp64 pixel directions of the camera (independent of the march)."""
    W, H = cam["width"], cam["height"]
    i, j = np.meshgrid(np.arange(W), np.arange(H))
    sx = (i + 0.5 - W / 2) * cam["pix"]
    sy = (H / 2 - j - 0.5) * cam["pix"]
    d = (np.array(cam["fwd"])[None, None] + sx[..., None] * np.array(cam["right"])[None, None]
         + sy[..., None] * np.array(cam["up"])[None, None])
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def test_raymarch_uniform_volume_closed_form():
    """One segment of colour (r, g, b, a): every sample has that value, so
    after the march A = 1 - (1 - a)^K and C = (r, g, b) * A, where K is the
    number of base steps covered, the ray's length in the volume over the
    base step (the lattice ends within one step of the exit)."""
    dims = (20, 14, 9)
    vol = np.zeros(dims[::-1], np.uint16)
    g = oracle.Graph(vol, 1)
    rgba = np.array([[0.2, 0.5, 0.9, 0.01]], np.float32)
    vals = np.repeat(rgba, g.N, axis=0)
    cam = _march_cam([-15.0, 3.0, 2.0], target=[10.0, 7.0, 4.5])
    img, steps, _ = g.raymarch(vals, cam)
    d = _ray_dirs(cam)
    eye = np.array(cam["eye"], np.float64)
    with np.errstate(divide="ignore"):
        t0 = (0.0 - eye) / d
        t1 = (np.array(dims, np.float64) - eye) / d
    tmin = np.minimum(t0, t1).max(axis=-1)
    tmax = np.maximum(t0, t1).min(axis=-1)
    hit = tmax > np.maximum(tmin, 0)
    assert hit.sum() > 50
    A = img[..., 3].astype(np.float64)
    assert (A[~hit] == 0).all() and (steps[~hit] == 0).all()
    # level 0 only (LOD bias -64): one sample per base step
    n = np.ceil((tmax - np.maximum(tmin, 0)) / cam["base_step"] - 1e-4)
    assert (np.abs(steps[hit] - n[hit]) <= 1).all()
    K = np.log1p(-A[hit]) / np.log1p(-0.01)
    assert np.allclose(K, steps[hit], atol=1e-2)
    for c in range(3):
        assert np.allclose(img[..., c][hit], rgba[0, c] * A[hit], rtol=1e-5)


def test_raymarch_opacity_correction_with_lod_steps():
    """With the LOD bias raised the march takes steps of 2^m base steps and
    corrects each sample's opacity to 1 - (1 - a)^(2^m): the total is still
    1 - (1 - a)^K with K the base steps covered."""
    dims = (64, 64, 64)
    vol = np.zeros(dims[::-1], np.uint16)
    g = oracle.Graph(vol, 1)
    vals = np.repeat(np.array([[0.3, 0.3, 0.3, 0.004]], np.float32), g.N, axis=0)
    cam0 = _march_cam([-40.0, 30.0, 31.0], target=[32.0, 32.0, 32.0], bias=-64)
    cam1 = dict(cam0, lod_bias=9)
    img0, st0, _ = g.raymarch(vals, cam0)
    img1, st1, _ = g.raymarch(vals, cam1)
    hit = st0 > 0
    assert (st1[hit] < st0[hit]).all()          # fewer, longer steps
    K0 = np.log1p(-img0[..., 3][hit].astype(np.float64)) / np.log1p(-0.004)
    K1 = np.log1p(-img1[..., 3][hit].astype(np.float64)) / np.log1p(-0.004)
    # the coarse march covers the same length up to its last (longest) step
    assert (np.abs(K1 - K0) <= 2 ** 6 + 1).all()
    assert np.allclose(K0, np.round(K0), atol=2e-2)
    assert np.allclose(K1, np.round(K1), atol=2e-1)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("bias", [-64, 9])
def test_raymarch_interpolation_reproduces_a_linear_field(axis, bias):
    """Segment ID = the voxel's coordinate along one axis, TF red = (ID + 1/2)
    / n: the field is linear in the voxel centres, every mip level holds its
    block averages (linear again), so trilinear and level interpolation give
    red = p / n exactly at interior points.  A single sample at the eye (ray
    parameter 0) reads that point; red / A recovers it."""
    dims = [16, 16, 16]
    n = dims[axis]
    coords = np.indices(dims[::-1])[2 - axis]
    vol = coords.astype(np.uint16)
    g = oracle.Graph(vol, n)
    tf = np.zeros((n, 4), np.float64)
    tf[:, 0] = (np.arange(n) + 0.5) / n
    tf[:, 3] = 0.5
    vals = oracle.propagate(g.p, g.q, g.a, g.b, n, tf).astype(np.float32)
    rng = np.random.default_rng(axis)
    for _ in range(6):
        eye = rng.uniform(5.0, 11.0, 3)
        cam = _march_cam(eye, width=2, height=2, bias=bias, max_steps=1)
        img, steps, _ = g.raymarch(vals, cam)
        assert (steps == 1).all()
        red = img[..., 0] / img[..., 3]
        assert np.allclose(red, np.float32(eye[axis]) / n, atol=2e-6), (eye, red)


def test_raymarch_skipping_changes_nothing():
    """Empty-space skipping only passes over samples of exactly zero opacity:
    the image is identical with and without it, and fewer samples are taken."""
    dims = (64, 64, 64)
    S = 4
    vol = synth.make_volume(4, dims=dims, S=S)   # three cylinders in a background (ID 0)
    g = oracle.Graph(vol, S)
    tf = synth.make_attribute_tf(4, S)           # background fully transparent
    vals = oracle.propagate(g.p, g.q, g.a, g.b, S, tf.astype(np.float64)).astype(np.float32)
    cam = synth.orbit_camera(4, dims=dims, width=48, height=32, base_step=0.5, lod_bias=0, ert=2.0)
    a, sa, _ = g.raymarch(vals, cam)
    b, sb, _ = g.raymarch(vals, cam, opacity=vals[:, 3].copy())
    assert np.array_equal(a, b)
    assert (sb <= sa).all() and sb.sum() < sa.sum()


# ---------------------------------------------------------------------------
# Sec. 3.3, Table 1: the bitstream
# ---------------------------------------------------------------------------
class _BitReader:
    """Fields least significant bit first, bit i of the stream = bit i % 8 of
    byte i / 8 (a reader written from Table 1's field list)."""

    def __init__(self, data):
        self.x = int.from_bytes(data, "little")
        self.pos = 0

    def get(self, n):
        v = (self.x >> self.pos) & ((1 << n) - 1)
        self.pos += n
        return v


def _read_stream(data, L):
    r = _BitReader(data)
    h = dict(S=r.get(32), fractional=r.get(1), nb=r.get(6) + 1, sigma_max=r.get(32),
             dims=[r.get(32) for _ in range(3)], bitrate=r.get(4) + 1)
    h["internal"] = r.get(h["nb"])
    h["exact"] = r.get(1)
    h["wbits"] = r.get(6) + 1
    h["r"], h["imin"] = [], []
    for _ in range(L):
        h["r"].append(r.get(h["nb"]))
        h["imin"].append(r.get(h["nb"]))
    h["header_bits"] = r.pos
    return h, r


@pytest.mark.parametrize("dims,S", [((37, 29, 23), 24), ((16, 16, 16), 1), ((9, 5, 3), 40)])
def test_bitstream_reads_back_the_graph(dims, S):
    vol = synth.make_volume(1, dims=dims, S=S) if S > 1 else np.zeros(dims[::-1], np.uint16)
    g = oracle.Graph(vol, S)
    data = g.bitstream()
    assert len(data) % 8 == 0
    h, r = _read_stream(data, g.L)
    assert h["S"] == S and h["fractional"] == 0 and h["exact"] == 1 and h["sigma_max"] == 0
    assert h["dims"] == list(dims) and h["internal"] == g.N - S
    assert h["nb"] == max(1, int(np.ceil(np.log2(g.N))))
    total = h["header_bits"]
    for l in range(g.L):
        ids = g.mip(l).ravel().astype(np.int64)
        lo, hi = ids.min(), ids.max()
        # Eq. 14-15: the smallest ID referenced and the bits of the range
        assert h["imin"][l] == lo
        assert h["r"][l] == int(np.ceil(np.log2(hi - lo + 1))) if hi > lo else h["r"][l] == 0
        got = np.array([r.get(h["r"][l]) for _ in range(ids.size)], np.int64) + lo
        assert np.array_equal(got, ids), l
        total += ids.size * h["r"][l]
    wmax = int(max(g.a[S:g.N].max(initial=1), g.b[S:g.N].max(initial=1)))
    assert h["wbits"] == max(1, wmax.bit_length())
    for n in range(S, g.N):
        assert (r.get(h["nb"]), r.get(h["nb"]), r.get(h["wbits"]), r.get(h["wbits"])) == \
            (g.p[n], g.q[n], g.a[n], g.b[n])
    total += (g.N - S) * 2 * (h["nb"] + h["wbits"])
    assert r.pos == total and len(data) == ((total + 7) // 8 + 7) // 8 * 8
    assert int.from_bytes(data, "little") >> total == 0    # zero padding


# ---------------------------------------------------------------------------
# Sec. 3.3 (Eq. 10-13), Sec. 3.7: greedy factorisation and the quantiser
# ---------------------------------------------------------------------------
def test_greedy_hand_worked_phi1():
    """Mixtures A = {1:1, 2:1, 3:2}, B = {1:1, 2:1}, C = {2:1, 3:1}.  phi_1:
    (1,2) and (2,3) occur in two mixtures each -> the smaller (1,2) first, and
    both occurrences give the same 1:1 lerp n4; then (2,3) and (3,n4) tie at
    one -> (2,3) (n5), then (3,n4) (n6, 2:2)."""
    g, roots, picks = oracle.greedy_lists([[(1, 1), (2, 1), (3, 2)], [(1, 1), (2, 1)], [(2, 1), (3, 1)]], 4,
                                          "occurrence", tau=1, bitrate=0)
    assert picks.tolist() == [[1, 2], [2, 3], [3, 4]]
    assert g.N == 7 and g.D == 2
    assert list(zip(g.p[4:7], g.q[4:7], g.a[4:7], g.b[4:7])) == [(1, 2, 1, 1), (2, 3, 1, 1), (3, 4, 1, 1)]
    assert roots.tolist() == [6, 4, 5]


def test_greedy_strategies_differ():
    """Two mixtures of five components and three of the pair {1, 2}: phi_1
    counts (1,2) three times against two for any pair of the large ones;
    phi_2 weighs each large mixture |h| - 1 = 4 (8 per pair) against 2 per
    small one (6): max-occurrence picks (1,2), max-reduction (3,4)."""
    big = [(i, 1) for i in range(3, 8)]
    lists = [big, big, [(1, 1), (2, 1)], [(1, 1), (2, 1)], [(1, 1), (2, 1)]]
    _, _, p1 = oracle.greedy_lists(lists, 8, "occurrence", tau=1)
    _, _, p2 = oracle.greedy_lists(lists, 8, "reduction", tau=1)
    assert p1[0].tolist() == [1, 2] and p2[0].tolist() == [3, 4]


def test_greedy_tau_skips_small_mixtures():
    vol = synth.make_volume(1, dims=(20, 17, 13), S=12)
    g, _, _, picks = oracle.greedy(vol, 12, "reduction", tau=64, bitrate=0)
    assert len(picks) == 0                       # nothing has more than 64 components
    g3, _, _, picks3 = oracle.greedy(vol, 12, "reduction", tau=3, bitrate=0)
    assert len(picks3) > 0


@pytest.mark.parametrize("strategy", ["occurrence", "reduction"])
def test_greedy_exact_mode_expands_to_every_mixture(strategy):
    """Without the quantiser every voxel's node expands exactly to its Eq. 4
    mixture, whatever the pick order."""
    dims = (21, 14, 11)
    vol = synth.make_volume(2, dims=dims, S=15)
    g, _, _, picks = oracle.greedy(vol, 15, strategy, tau=3, bitrate=0)
    assert len(picks) > 0
    for l in range(1, g.L):
        off, ids, cnt = oracle.mixtures(vol, l)
        mip = g.mip(l).ravel()
        for v in range(len(mip)):
            total = int(cnt[off[v]:off[v + 1]].sum())
            e = oracle.expand(g.p, g.q, g.a, g.b, 15, int(mip[v]), total)
            want = np.zeros(15, np.uint64)
            want[ids[off[v]:off[v + 1]]] = cnt[off[v]:off[v + 1]]
            assert np.array_equal(e, want), (l, v)


@pytest.mark.parametrize("bitrate", [3, 6, 9])
def test_greedy_quantiser_error_bound(bitrate):
    """Each lerp's weight is off by at most half a bin (2^-(b+1)); pushing a
    unit of mass through a tree moves at most twice that per level, so every
    reconstructed mixture is within D * 2^-b of Eq. 4 in l1, and still sums
    to 1.  Codewords are the bin centres; sigma lies within half a bin."""
    dims = (24, 20, 16)
    vol = synth.make_volume(1, dims=dims, S=20)
    g, cb, sg, _ = oracle.greedy(vol, 20, "reduction", tau=3, bitrate=bitrate)
    nb = 1 << bitrate
    assert np.allclose(cb, (2 * np.arange(nb) + 1) / (2.0 * nb))
    assert (sg >= 0).all() and (sg <= 0.5 / nb + 1e-12).all() and (sg > 0).any()
    assert (g.a[20:g.N] < nb).all() and (g.b[20:g.N] == 0).all()
    worst = 0.0
    for l in range(1, g.L):
        off, ids, cnt = oracle.mixtures(vol, l)
        mip = g.mip(l).ravel()
        for v in range(0, len(mip), 7):
            rec = oracle.quantised_mixture(g, cb, int(mip[v]))
            h = np.zeros(20)
            c = cnt[off[v]:off[v + 1]].astype(np.float64)
            h[ids[off[v]:off[v + 1]]] = c / c.sum()
            assert abs(rec.sum() - 1.0) < 1e-12
            worst = max(worst, np.abs(rec - h).sum())
    assert worst <= g.D * 2.0 ** -bitrate


def test_greedy_coarser_bins_reuse_more():
    vol = synth.make_volume(1, dims=(32, 32, 32), S=24)
    n = [oracle.greedy(vol, 24, "reduction", tau=3, bitrate=b)[0].N for b in (3, 9, 0)]
    assert n[0] <= n[1] <= n[2]


# ---------------------------------------------------------------------------
# Sec. 3.5 (Eq. 16-17): error propagation through the mixture table
# ---------------------------------------------------------------------------
def test_error_rows_closed_form_of_two_lerps():
    """n4 = lerp(e0, e1; w = 1/4), n5 = lerp(n4, e2; w = 1/2), weight
    uncertainties 0.01 and 0.02.  Eq. 17: n4's components carry relative
    error sqrt(2) * 0.01 / (1/4); n5 adds 2 (0.02 / (1/2))^2 to the squared
    relative error of the components from n4, and e2 gets that term alone."""
    g, _ = oracle.factor_lists([[(0, 3), (1, 1)], [(0, 3), (1, 1), (2, 4)]], 3)
    # the pairwise rule: n3 = (e0, e1, 3:1), n4 = (n3, e2, 4:4)
    assert g.N == 5 and list(g.p[3:5]) == [0, 3] and list(g.q[3:5]) == [1, 2]
    w = np.array([0, 0, 0, 0.25, 0.5]); dw = np.array([0, 0, 0, 0.01, 0.02])
    off, src, mu, dmu = oracle.error_rows(g, w, dw)
    r3 = slice(off[3], off[4]); r4 = slice(off[4], off[5])
    assert src[r3].tolist() == [0, 1] and np.allclose(mu[r3], [0.75, 0.25])
    rel3 = np.sqrt(2) * 0.01 / 0.25
    assert np.allclose(dmu[r3], np.array([0.75, 0.25]) * rel3)
    assert src[r4].tolist() == [0, 1, 2] and np.allclose(mu[r4], [0.375, 0.125, 0.5])
    rel4 = np.sqrt(rel3 ** 2 + 2 * (0.02 / 0.5) ** 2)
    assert np.allclose(dmu[r4], [0.375 * rel4, 0.125 * rel4, 0.5 * np.sqrt(2) * 0.04])


def test_error_rows_match_the_tree_pushes_and_exact_graphs_have_none():
    vol = synth.make_volume(1, dims=(24, 20, 16), S=20)
    gq, cb, sg, _ = oracle.greedy(vol, 20, "reduction", tau=3, bitrate=6)
    off, src, mu, dmu = oracle.error_rows(gq, *oracle.node_weights(gq, cb, sg))
    for n in range(20, gq.N, 37):
        dense = np.zeros(20)
        sl = slice(off[n], off[n + 1])
        dense[src[sl]] = mu[sl]
        assert np.allclose(dense, oracle.quantised_mixture(gq, cb, n), rtol=1e-12, atol=1e-15)
    assert (dmu[off[20]:] > 0).any()
    ge = oracle.Graph(vol, 20)
    _, _, _, dmu_e = oracle.error_rows(ge, *oracle.node_weights(ge))
    assert (dmu_e == 0).all()


def test_lut_query_exact_counts_and_error_bars():
    """Exact graphs: the table's sums are the brute-force counts.  Quantised
    graphs: the sums still add up to the box volume (convex lerps), and the
    error bar of a one-cube box is its node's Eq. 17 uncertainty times 8^l."""
    dims = (24, 20, 16)
    vol = synth.make_volume(1, dims=dims, S=20)
    boxes = synth.make_boxes(1, Q=60, dims=dims, box_max=24)
    ge = oracle.Graph(vol, 20)
    h, e = oracle.lut_query(ge, oracle.error_rows(ge, *oracle.node_weights(ge)), boxes)
    assert np.allclose(h, oracle.box_hist(vol, 20, boxes), rtol=1e-12, atol=1e-9) and (e == 0).all()
    gq, cb, sg, _ = oracle.greedy(vol, 20, "reduction", tau=3, bitrate=5)
    rows = oracle.error_rows(gq, *oracle.node_weights(gq, cb, sg))
    hq, eq = oracle.lut_query(gq, rows, boxes)
    vq = np.prod(np.minimum(boxes[:, :3] + boxes[:, 3:], dims) - boxes[:, :3], axis=1)
    assert np.allclose(hq.sum(axis=1), vq, rtol=1e-12)
    one = np.array([[8, 4, 4, 4, 4, 4]], np.int32)          # a single level-2 cube
    h1, e1 = oracle.lut_query(gq, rows, one)
    off, src, mu, dmu = rows
    node = int(gq.mip(2)[1, 1, 2])
    sl = slice(off[node], off[node + 1])
    want = np.zeros(20)
    want[src[sl]] = 64 * dmu[sl]
    assert np.allclose(e1[0], want)
