"""CPU oracle for the Mixture Graph hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct statement of what the GPU library computes,
in exact integers and fp64 (see ``mg_oracle.c`` for the passage of the paper
each function follows and for the readings taken where the paper is silent).
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Functions whose results are pinned by tests other than self-comparison:
  level_dims        Table 2 voxel totals and level counts; hand cases
  mixtures          Eq. 1-2 invariants, hand volumes, level-0 losslessness
  build             paper Fig. 4 re-use; expansion equals the mixtures (Eq. 4)
  expand            rational expansion of the paper's Fig. 2 / Fig. 4 examples
  propagate         direct convex combination; unit-vector TF gives mixtures
  box_hist          brute force, a plain count; sum equals the clipped volume
  fa_cubes          brute-force tiling of the clipped box; Table 3 arithmetic
  fa_query          equals box_hist exactly
  sample_voxels     hand cases at level and voxel boundaries
  raymarch          closed form through a uniform volume; exact trilinear
                    reproduction of a linear field; skipping changes nothing
  bitstream         read back by an independent reader of Table 1's layout;
                    section sizes from Eq. 15
  error_rows        a lerp's closed form (Eq. 17); rows equal the tree pushes;
                    zero uncertainty for exact weights
  lut_query         equals box_hist for exact graphs; error bars by Eq. 16
  greedy            hand-worked picks (phi_1 and phi_2 differ); exact mode
                    expands to every mixture; quantisation error within its
                    bound; codewords and sigma by definition
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmg_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 40
NONE = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, fp contraction off, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fopenmp",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _LevelOut(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("off", ctypes.POINTER(ctypes.c_uint64)),
                ("ids", ctypes.POINTER(ctypes.c_uint32)),
                ("cnt", ctypes.POINTER(ctypes.c_uint64))]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        lib.mgo_level_dims.argtypes = [i64, i64, i64, P, i32]
        lib.mgo_level_dims.restype = i32
        lib.mgo_mixtures.argtypes = [P, i32, i64, i64, i64, i32, ctypes.POINTER(_LevelOut)]
        lib.mgo_mixtures.restype = i32
        lib.mgo_level_release.argtypes = [ctypes.POINTER(_LevelOut)]
        lib.mgo_build.argtypes = [P, i32, i64, i64, i64, ctypes.c_uint32]
        lib.mgo_build.restype = P
        lib.mgo_graph_free.argtypes = [P]
        for name, rt in (("mgo_graph_nodes", i64), ("mgo_graph_depth", i32),
                         ("mgo_graph_levels", i32), ("mgo_graph_max_nnz", i64),
                         ("mgo_graph_pairs", i64)):
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = rt
        lib.mgo_graph_dims.argtypes = [P, P]
        lib.mgo_graph_nodes_copy.argtypes = [P, P, P, P, P, P]
        lib.mgo_graph_buckets_copy.argtypes = [P, P]
        lib.mgo_graph_mip_copy.argtypes = [P, i32, P]
        lib.mgo_expand.argtypes = [P, P, P, P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, P]
        lib.mgo_expand.restype = i32
        lib.mgo_propagate.argtypes = [P, P, P, P, i64, ctypes.c_uint32, P, i32, P]
        lib.mgo_direct_colors.argtypes = [P, P, P, i64, P, i32, P]
        lib.mgo_box_hist.argtypes = [P, i32, i64, i64, i64, ctypes.c_uint32, P, i64, P]
        lib.mgo_footprint_1d.argtypes = [i64, i64, i64, P]
        lib.mgo_footprint_1d.restype = i32
        lib.mgo_fa_cubes.argtypes = [P, i64, i64, i64, P, i64]
        lib.mgo_fa_cubes.restype = i64
        lib.mgo_fa_query.argtypes = [P, P, i64, P]
        lib.mgo_fa_query.restype = i32
        lib.mgo_sample_voxels.argtypes = [P, i32, P, i64, P, P]
        lib.mgo_factor_lists.argtypes = [P, P, P, i64, ctypes.c_uint32, P]
        lib.mgo_factor_lists.restype = P
        lib.mgo_depths.argtypes = [P, P, i64, ctypes.c_uint32, P]
        lib.mgo_raymarch.argtypes = [P, P, P, ctypes.POINTER(Camera), P, P, P]
        lib.mgo_build_greedy.argtypes = [P, i32, i64, i64, i64, ctypes.c_uint32, i32, i32, i32, P, P, P, i64, P]
        lib.mgo_build_greedy.restype = P
        lib.mgo_greedy_lists.argtypes = [P, P, P, i64, ctypes.c_uint32, i32, i32, i32, P, P, i64, P]
        lib.mgo_greedy_lists.restype = P
        lib.mgo_quantised_mixture.argtypes = [P, P, ctypes.c_uint32, P]
        lib.mgo_error_rows.argtypes = [P, P, P, P, i64, ctypes.c_uint32, P, P, P, P]
        lib.mgo_error_rows.restype = i32
        lib.mgo_lut_query.argtypes = [P, P, P, P, P, P, i64, P, P]
        lib.mgo_bitstream.argtypes = [P, P, i64]
        lib.mgo_bitstream.restype = i64
        lib.mgo_set_threads.argtypes = [i32]
        lib.mgo_set_threads.restype = i32
        _lib = lib
        return lib


class Camera(ctypes.Structure):
    """Pinhole camera and march settings of raymarch (Sec. 4): eye and an
    orthonormal basis (fwd, right, up) in level-0 voxel units, the angle of a
    pixel, the image size, the lattice step (level-0 voxels), an integer LOD
    bias, the early-termination opacity (> 1: none) and a step cap."""
    _fields_ = [("eye", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("pix", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("base_step", ctypes.c_float), ("lod_bias", ctypes.c_int32),
                ("ert", ctypes.c_float), ("max_steps", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


def camera(cam: dict) -> Camera:
    c = Camera()
    for k in ("eye", "fwd", "right", "up"):
        for i in range(3):
            getattr(c, k)[i] = float(np.float32(cam[k][i]))
    c.pix = float(np.float32(cam["pix"]))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.base_step = float(np.float32(cam["base_step"]))
    c.lod_bias = int(cam["lod_bias"])
    c.ert = float(np.float32(cam["ert"]))
    c.max_steps = int(cam["max_steps"])
    return c


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return ctypes.c_void_p(a.ctypes.data)


def _vol_args(vol: np.ndarray):
    vol = np.ascontiguousarray(vol)
    if vol.dtype == np.uint16:
        nb = 2
    elif vol.dtype == np.uint32:
        nb = 4
    else:
        raise TypeError("volume must be uint16 or uint32")
    nz, ny, nx = vol.shape
    return vol, nb, nx, ny, nz


# --------------------------------------------------------------------------
# Eq. 4 (Sec. 3.1): level geometry
# --------------------------------------------------------------------------
def level_dims(nx: int, ny: int, nz: int) -> np.ndarray:
    """(L, 3) array of per-level (x, y, z) resolutions, level 0 first."""
    out = np.zeros(MAX_LEVELS * 3, dtype=np.int64)
    L = _load().mgo_level_dims(nx, ny, nz, _ptr(out), MAX_LEVELS)
    if L < 1:
        raise ValueError("invalid dims")
    return out[: 3 * L].reshape(L, 3).copy()


# --------------------------------------------------------------------------
# Eq. 4: integer mixture lists of one level (c = 8^l * H)
# --------------------------------------------------------------------------
def mixtures(vol: np.ndarray, level: int):
    """Returns (off u64[V+1], ids u32[nnz], cnt u64[nnz]) for one level."""
    vol, nb, nx, ny, nz = _vol_args(vol)
    lo = _LevelOut()
    rc = _load().mgo_mixtures(_ptr(vol), nb, nx, ny, nz, level, ctypes.byref(lo))
    if rc:
        raise MemoryError("oracle mixtures failed")
    try:
        off = np.ctypeslib.as_array(lo.off, shape=(lo.nv + 1,)).copy()
        ids = np.ctypeslib.as_array(lo.ids, shape=(max(lo.nnz, 1),))[: lo.nnz].copy()
        cnt = np.ctypeslib.as_array(lo.cnt, shape=(max(lo.nnz, 1),))[: lo.nnz].copy()
    finally:
        _load().mgo_level_release(ctypes.byref(lo))
    return off, ids, cnt


# --------------------------------------------------------------------------
# Sec. 3.2-3.4: the Mixture Graph (canonical numbering)
# --------------------------------------------------------------------------
class Graph:
    """Oracle Mixture Graph: node table in canonical order and mip IDs."""

    def __init__(self, vol: np.ndarray, num_segments: int, _handle=None):
        lib = _load()
        if _handle is None:
            vol, nb, nx, ny, nz = _vol_args(vol)
            h = lib.mgo_build(_ptr(vol), nb, nx, ny, nz, num_segments)
            if not h:
                raise ValueError("oracle build failed (ID >= num_segments or out of memory)")
        else:
            h = _handle
        self._h = h
        self._lib = lib
        self.S = int(num_segments)
        self.N = int(lib.mgo_graph_nodes(h))
        self.D = int(lib.mgo_graph_depth(h))
        self.L = int(lib.mgo_graph_levels(h))
        self.max_nnz = int(lib.mgo_graph_max_nnz(h))
        self.pairs = int(lib.mgo_graph_pairs(h))
        dims = np.zeros(max(self.L, 1) * 3, dtype=np.int64)
        if self.L:
            lib.mgo_graph_dims(h, _ptr(dims))
        self.dims = dims[: 3 * self.L].reshape(self.L, 3)
        n = max(self.N, 1)
        self.p = np.zeros(n, np.uint32)
        self.q = np.zeros(n, np.uint32)
        self.a = np.zeros(n, np.uint64)
        self.b = np.zeros(n, np.uint64)
        self.depth = np.zeros(n, np.int32)
        lib.mgo_graph_nodes_copy(h, _ptr(self.p), _ptr(self.q), _ptr(self.a), _ptr(self.b),
                                 _ptr(self.depth))
        self.bucket = np.zeros(self.D + 2, np.int64)
        lib.mgo_graph_buckets_copy(h, _ptr(self.bucket))
        self._vol = vol

    def mip(self, level: int) -> np.ndarray:
        """Canonical node ID of every voxel of one level, shape (z, y, x)."""
        d = self.dims[level]
        out = np.zeros(int(d[0] * d[1] * d[2]), np.uint32)
        self._lib.mgo_graph_mip_copy(self._h, level, _ptr(out))
        return out.reshape(int(d[2]), int(d[1]), int(d[0]))

    def raymarch(self, vals: np.ndarray, cam: dict, opacity: np.ndarray = None):
        """One RGBA image (H, W, 4) fp32 marched through node values vals
        (N, 4) fp32 (Sec. 4); with opacity (N,) fp32, empty space is skipped.
        Returns (image, samples per pixel, smallest |A - ert| per pixel)."""
        vals = np.ascontiguousarray(vals, np.float32).reshape(self.N, 4)
        op = None if opacity is None else np.ascontiguousarray(opacity, np.float32).reshape(self.N)
        c = camera(cam)
        img = np.zeros((c.height, c.width, 4), np.float32)
        steps = np.zeros((c.height, c.width), np.int32)
        margin = np.zeros((c.height, c.width), np.float32)
        self._lib.mgo_raymarch(self._h, _ptr(vals), None if op is None else _ptr(op), ctypes.byref(c), _ptr(img),
                               _ptr(steps), _ptr(margin))
        return img, steps, margin

    def bitstream(self) -> bytes:
        """The graph as the bitstream of Table 1 (Sec. 3.3, Eq. 14-15), exact
        weights in the extension field (see mg_oracle.c for the readings)."""
        n = int(self._lib.mgo_bitstream(self._h, None, 0))
        out = np.zeros(max(n, 8), np.uint8)
        self._lib.mgo_bitstream(self._h, _ptr(out), out.nbytes)
        return out[:n].tobytes()

    def fa_query(self, boxes: np.ndarray) -> np.ndarray:
        """Box histograms by footprint assembly + exact push (Algorithm 1)."""
        boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 6)
        out = np.zeros((boxes.shape[0], self.S), np.uint32)
        rc = self._lib.mgo_fa_query(self._h, _ptr(boxes), boxes.shape[0], _ptr(out))
        if rc:
            raise ArithmeticError("inexact division in the push")
        return out

    def close(self):
        if self._h:
            self._lib.mgo_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def factor_lists(lists, num_segments: int):
    """Factorise given mixtures (Sec. 3.2) with the oracle's rule.

    lists: sequence of [(segment id, integer weight), ...] sorted by id.
    Returns (Graph without mip levels, roots) where roots[m] is the canonical
    node representing mixture m."""
    off = [0]
    ids, cnt = [], []
    for lst in lists:
        for sid, w in lst:
            ids.append(int(sid)); cnt.append(int(w))
        off.append(len(ids))
    off = np.array(off, np.uint64)
    ids = np.array(ids if ids else [0], np.uint32)
    cnt = np.array(cnt if cnt else [0], np.uint64)
    roots = np.zeros(max(len(lists), 1), np.uint32)
    h = _load().mgo_factor_lists(_ptr(off), _ptr(ids), _ptr(cnt), len(lists), num_segments,
                                 _ptr(roots))
    if not h:
        raise MemoryError("oracle factorisation failed")
    return Graph(None, num_segments, _handle=h), roots[: len(lists)]


STRATEGIES = {"occurrence": 1, "reduction": 2}   # phi_1 max-occurrence, phi_2 max-reduction (Eq. 10-13)


def greedy(vol: np.ndarray, num_segments: int, strategy: str = "reduction", tau: int = 3, bitrate: int = 9,
           max_picks: int = 1 << 16):
    """Greedy factorisation of a volume's mipmap (Sec. 3.3, Sec. 3.7): returns
    (Graph, codebook (2^b,), sigma (2^b,), stage-1 picks (n, 2)).  bitrate 0
    keeps exact ratios (then a, b are the exact weights); otherwise a node's
    `a` is its quantiser bin and b = 0."""
    vol, nb, nx, ny, nz = _vol_args(vol)
    nbins = (1 << bitrate) if bitrate else 1
    cb = np.zeros(nbins, np.float64)
    sg = np.zeros(nbins, np.float64)
    picks = np.zeros((max_picks, 2), np.uint32)
    n = ctypes.c_int64(0)
    h = _load().mgo_build_greedy(_ptr(vol), nb, nx, ny, nz, num_segments, STRATEGIES[strategy], tau, bitrate,
                                 _ptr(cb), _ptr(sg), _ptr(picks), max_picks, ctypes.byref(n))
    if not h:
        raise ValueError("oracle greedy build failed")
    g = Graph(None, num_segments, _handle=h)
    return g, cb, sg, picks[: min(n.value, max_picks)].copy()


def greedy_lists(lists, num_segments: int, strategy: str = "reduction", tau: int = 3, bitrate: int = 0,
                 max_picks: int = 1024):
    """Greedy factorisation of given mixtures [(id, weight), ...] ascending by
    id: returns (Graph, roots, stage-1 picks)."""
    off = [0]
    ids, cnt = [], []
    for lst in lists:
        for sid, w in lst:
            ids.append(int(sid)); cnt.append(int(w))
        off.append(len(ids))
    off = np.array(off, np.uint64)
    ids = np.array(ids if ids else [0], np.uint32)
    cnt = np.array(cnt if cnt else [0], np.uint64)
    roots = np.zeros(max(len(lists), 1), np.uint32)
    picks = np.zeros((max_picks, 2), np.uint32)
    n = ctypes.c_int64(0)
    h = _load().mgo_greedy_lists(_ptr(off), _ptr(ids), _ptr(cnt), len(lists), num_segments, STRATEGIES[strategy],
                                 tau, bitrate, _ptr(roots), _ptr(picks), max_picks, ctypes.byref(n))
    if not h:
        raise ValueError("oracle greedy failed")
    return Graph(None, num_segments, _handle=h), roots[: len(lists)], picks[: min(n.value, max_picks)].copy()


def quantised_mixture(g, codebook: np.ndarray, node: int) -> np.ndarray:
    """The mixture (S,) a quantised graph reconstructs for one node."""
    cb = np.ascontiguousarray(codebook, np.float64)
    out = np.zeros(g.S, np.float64)
    _load().mgo_quantised_mixture(g._h, _ptr(cb), int(node), _ptr(out))
    return out


def node_weights(g, codebook=None, sigma=None):
    """(w, dw) of every node (Sec. 3.5): the weight of q and its uncertainty;
    exact graphs b/(a+b) and 0, quantised graphs their bin's codeword and
    sigma.  Sources get 0, 0."""
    N, S = g.N, g.S
    w = np.zeros(N, np.float64)
    dw = np.zeros(N, np.float64)
    if codebook is None:
        a = g.a[S:N].astype(np.float64); b = g.b[S:N].astype(np.float64)
        w[S:] = b / (a + b)
    else:
        k = g.a[S:N].astype(np.int64)
        w[S:] = np.asarray(codebook, np.float64)[k]
        dw[S:] = np.asarray(sigma, np.float64)[k]
    return w, dw


def error_rows(g, w, dw):
    """Every node's mixture with its Eq. 17 uncertainty: (off (N+1,), src,
    mu, dmu); row n is [off[n], off[n+1]), sources ascending (unused slack
    entries hold source 2^32 - 1)."""
    P_, Q_ = np.ascontiguousarray(g.p[:g.N]), np.ascontiguousarray(g.q[:g.N])
    w = np.ascontiguousarray(w, np.float64); dw = np.ascontiguousarray(dw, np.float64)
    off = np.zeros(g.N + 1, np.int64)
    lib = _load()
    if lib.mgo_error_rows(_ptr(P_), _ptr(Q_), _ptr(w), _ptr(dw), g.N, g.S, _ptr(off), None, None, None):
        raise ValueError("malformed node table")
    E = int(off[-1])
    src = np.zeros(max(E, 1), np.uint32); mu = np.zeros(max(E, 1)); dmu = np.zeros(max(E, 1))
    lib.mgo_error_rows(_ptr(P_), _ptr(Q_), _ptr(w), _ptr(dw), g.N, g.S, _ptr(off), _ptr(src), _ptr(mu), _ptr(dmu))
    return off, src[:E], mu[:E], dmu[:E]


def lut_query(g, rows, boxes):
    """Box histograms summed from the mixture table (Sec. 3.6) and their
    error bars (Sec. 3.5): ((Q, S) expected counts, (Q, S) error bars)."""
    off, src, mu, dmu = (np.ascontiguousarray(x) for x in rows)
    boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 6)
    hist = np.zeros((boxes.shape[0], g.S)); err = np.zeros((boxes.shape[0], g.S))
    _load().mgo_lut_query(g._h, _ptr(off), _ptr(src), _ptr(mu), _ptr(dmu), _ptr(boxes), boxes.shape[0], _ptr(hist),
                          _ptr(err))
    return hist, err


def depths(p, q, S: int) -> np.ndarray:
    """Topological level of every node (Sec. 3.4, Fig. 5)."""
    p = np.ascontiguousarray(p, np.uint32); q = np.ascontiguousarray(q, np.uint32)
    out = np.zeros(p.shape[0], np.int32)
    _load().mgo_depths(_ptr(p), _ptr(q), p.shape[0], S, _ptr(out))
    return out


def expand(p, q, a, b, S: int, node: int, total: int) -> np.ndarray:
    """Exact integer expansion of one node: dense histogram of S counts that
    the total `total` splits into (Sec. 3.2 tree of lerps)."""
    p = np.ascontiguousarray(p, np.uint32); q = np.ascontiguousarray(q, np.uint32)
    a = np.ascontiguousarray(a, np.uint64); b = np.ascontiguousarray(b, np.uint64)
    out = np.zeros(S, np.uint64)
    rc = _load().mgo_expand(_ptr(p), _ptr(q), _ptr(a), _ptr(b), S, node, total, _ptr(out))
    if rc:
        raise ArithmeticError("inexact division while expanding node %d" % node)
    return out


def propagate(p, q, a, b, S: int, tf: np.ndarray) -> np.ndarray:
    """fp64 colour of every node (Sec. 3.4): TF at sources, lerps in ID order."""
    p = np.ascontiguousarray(p, np.uint32); q = np.ascontiguousarray(q, np.uint32)
    a = np.ascontiguousarray(a, np.uint64); b = np.ascontiguousarray(b, np.uint64)
    tf = np.ascontiguousarray(tf, np.float64)
    C = tf.shape[1]
    N = p.shape[0]
    out = np.zeros((N, C), np.float64)
    _load().mgo_propagate(_ptr(p), _ptr(q), _ptr(a), _ptr(b), N, S, _ptr(tf), C, _ptr(out))
    return out


def direct_colors(vol: np.ndarray, level: int, tf: np.ndarray) -> np.ndarray:
    """fp64 colour sum_i H_i TF(i) of every voxel of one level, (V, C)."""
    off, ids, cnt = mixtures(vol, level)
    tf = np.ascontiguousarray(tf, np.float64)
    C = tf.shape[1]
    nv = off.shape[0] - 1
    out = np.zeros((nv, C), np.float64)
    _load().mgo_direct_colors(_ptr(off), _ptr(ids), _ptr(cnt), nv, _ptr(tf), C, _ptr(out))
    return out


def box_hist(vol: np.ndarray, num_segments: int, boxes: np.ndarray) -> np.ndarray:
    """Brute-force box histograms (Q, S) uint32 over the level-0 IDs."""
    vol, nb, nx, ny, nz = _vol_args(vol)
    boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 6)
    out = np.zeros((boxes.shape[0], num_segments), np.uint32)
    _load().mgo_box_hist(_ptr(vol), nb, nx, ny, nz, num_segments, _ptr(boxes),
                         boxes.shape[0], _ptr(out))
    return out


def footprint_1d(i: int, di: int, dim: int) -> list:
    r = np.zeros(130, np.int32)
    n = _load().mgo_footprint_1d(i, di, dim, _ptr(r))
    return [int(v) for v in r[:n]]


def fa_cubes(box, nx: int, ny: int, nz: int) -> np.ndarray:
    """(n, 4) array of (level, x, y, z) for every cube of a box (Algorithm 1)."""
    box = np.ascontiguousarray(box, dtype=np.int32).reshape(6)
    lib = _load()
    n = lib.mgo_fa_cubes(_ptr(box), nx, ny, nz, None, 0)
    out = np.zeros((max(n, 1), 4), np.int32)
    lib.mgo_fa_cubes(_ptr(box), nx, ny, nz, _ptr(out), n)
    return out[:n]


def fa_count(box, nx: int, ny: int, nz: int) -> int:
    box = np.ascontiguousarray(box, dtype=np.int32).reshape(6)
    return int(_load().mgo_fa_cubes(_ptr(box), nx, ny, nz, None, 0))


def sample_voxels(dims: np.ndarray, samples: np.ndarray):
    """Level and linear voxel index of every (x, y, z, lod) sample (Sec. 4)."""
    dims = np.ascontiguousarray(dims, np.int64).reshape(-1, 3)
    samples = np.ascontiguousarray(samples, np.float32).reshape(-1, 4)
    P = samples.shape[0]
    lev = np.zeros(P, np.int32)
    vox = np.zeros(P, np.int64)
    _load().mgo_sample_voxels(_ptr(dims), dims.shape[0], _ptr(samples), P, _ptr(lev), _ptr(vox))
    return lev, vox


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (0: leave as is); returns the count in use."""
    return int(_load().mgo_set_threads(int(n)))
