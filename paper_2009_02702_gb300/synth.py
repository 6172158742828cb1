"""Seeded synthetic inputs shaped like the paper's data sets.

Input generation only: this module holds none of the Mixture Graph's
arithmetic, and both the GPU library's tests and the CPU oracle take their
inputs from here.  The paper's volumes (Hippocampus, Neocortex, Polymer,
Sec. 5 / Table 2) are not available; the recipes below reproduce their shapes,
segment counts and structure:

  cfg 1  64^3 uint16, 64 segments, Voronoi of uniform seeds
  cfg 2  512x512x384 uint16, 353 segments, Voronoi with power-law
         (Pareto alpha = 1.5) multiplicative seed weights (Hippocampus-like)
  cfg 3  2048x2048x300 uint16, 1,182 segments, Voronoi with cells stretched
         4x along z (Neocortex-like)
  cfg 4  614x961x600 uint16, background 0 plus 15,916 non-overlapping random
         cylinders, radius 2-6, length 50-600 (Polymer-like)
  cfg 5  serving mix over the volumes of cfgs 1-3: Poisson arrivals (mean
         20,000 requests/s), 90% box histograms with log-uniform sides, 10%
         TF frames

Every draw comes from numpy's PCG64 seeded with 2009027020 + config index
(one independent stream per purpose).  Voronoi assignment is exact integer
arithmetic (see csrc/synth_host.c), identical on the host and the GPU.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

BASE_SEED = 2009027020
_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")

# stream indices of the per-purpose generators
_STREAM_VOLUME, _STREAM_BOXES, _STREAM_TF, _STREAM_SAMPLES = 0, 1, 2, 3

CONFIGS = {
    1: dict(name="voronoi-64x64x64-s64", dims=(64, 64, 64), S=64, kind="voronoi",
            metric=(1, 1, 1), weighted=False, queries=1000, box="uniform", box_max=64),
    2: dict(name="voronoi-512x512x384-s353-powerlaw", dims=(512, 512, 384), S=353,
            kind="voronoi", metric=(1, 1, 1), weighted=True, queries=10000,
            box="loguniform", box_max=512),
    3: dict(name="voronoi-2048x2048x300-s1182-aniso4z", dims=(2048, 2048, 300), S=1182,
            kind="voronoi", metric=(16, 16, 1), weighted=False, queries=100000,
            box="loguniform", box_max=1024),
    4: dict(name="cylinders-614x961x600-s15917", dims=(614, 961, 600), S=15917,
            kind="cylinders", queries=10000, box="loguniform", box_max=600,
            radius=(2.0, 6.0), length=(50.0, 600.0), tries=32),
    5: dict(name="serving-mix-cfg1-3-poisson20k", volumes=(1, 2, 3), rate=20000.0, tf_frac=0.1,
            requests=200000, frame_samples=4096),
}


def rng_for(cfg_index: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([BASE_SEED + int(cfg_index), int(stream)]))


# --------------------------------------------------------------------------
# compiled helpers
# --------------------------------------------------------------------------
_host = None
_dev = None


def _host_lib():
    global _host
    if _host is None:
        path = os.path.join(_BUILD, "libmgsynth_host.so")
        if not os.path.exists(path):
            from . import build as _b
            _b.build_synth_host()
        lib = ctypes.CDLL(path)
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.mgs_voronoi.argtypes = [i64, i64, i64, P, P, i64, P, ctypes.c_int, P]
        lib.mgs_voronoi_block.argtypes = [i64, i64, i64, i64, i64, i64, P, P, i64, P, ctypes.c_int, P]
        lib.mgs_voronoi_block_brute.argtypes = lib.mgs_voronoi_block.argtypes
        lib.mgs_cylinders.argtypes = [i64, i64, i64, i64, i64, P, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, P]
        lib.mgs_cylinders.restype = i64
        _host = lib
    return _host


def _dev_lib():
    global _dev
    if _dev is None:
        path = os.path.join(_BUILD, "libmgsynth_dev.so")
        if not os.path.exists(path):
            raise RuntimeError("GPU volume generator not built: run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.mgs_voronoi_dev.argtypes = [i64, i64, i64, P, P, i64, P, ctypes.c_int, P, P]
        lib.mgs_voronoi_dev.restype = ctypes.c_int
        _dev = lib
    return _dev


# --------------------------------------------------------------------------
# Voronoi volumes
# --------------------------------------------------------------------------
def voronoi_seeds(dims, K: int, weighted: bool, rng: np.random.Generator):
    """Doubled seed coordinates (K, 3) int64 and integer weights (K,) int64.

    Weighted seeds draw w = U^(-1/1.5) (Pareto, alpha 1.5, x_m = 1) and the
    voxel goes to argmin |x - s_i| / w_i^(1/3), i.e. argmin d_i^2 / W_i with
    W_i = round(w_i^(2/3) * 2^16) clamped to [1, 2^31 - 1]."""
    nx, ny, nz = dims
    hi = np.array([2 * nx, 2 * ny, 2 * nz], dtype=np.int64)
    seeds2 = rng.integers(0, hi, size=(K, 3), dtype=np.int64)
    if weighted:
        u = 1.0 - rng.random(K)
        w = u ** (-1.0 / 1.5)
        W = np.rint(w ** (2.0 / 3.0) * 65536.0)
        W = np.clip(W, 1, 2 ** 31 - 1).astype(np.int64)
    else:
        W = np.ones(K, dtype=np.int64)
    return np.ascontiguousarray(seeds2), np.ascontiguousarray(W)


def voronoi_host(dims, seeds2, W, metric, dtype=np.uint16) -> np.ndarray:
    nx, ny, nz = dims
    out = np.zeros((nz, ny, nx), dtype=dtype)
    m = np.ascontiguousarray(np.array(metric, dtype=np.int64))
    _host_lib().mgs_voronoi(nx, ny, nz, seeds2.ctypes.data, W.ctypes.data, seeds2.shape[0],
                            m.ctypes.data, out.itemsize, out.ctypes.data)
    return out


def voronoi_window(cfg_index: int, origin, extent, dims=None, S=None) -> np.ndarray:
    """The (ez, ey, ex) block at voxel `origin` (x, y, z) of a Voronoi config's
    volume, generated on the host without the rest of the volume."""
    cfg = CONFIGS[cfg_index]
    dims = tuple(dims) if dims is not None else cfg["dims"]
    S = int(S) if S is not None else cfg["S"]
    seeds2, W = voronoi_seeds(dims, S, cfg["weighted"], rng_for(cfg_index, _STREAM_VOLUME))
    ex, ey, ez = (int(e) for e in extent)
    out = np.zeros((ez, ey, ex), dtype=np.uint16)
    m = np.ascontiguousarray(np.array(cfg["metric"], dtype=np.int64))
    _host_lib().mgs_voronoi_block(int(origin[0]), int(origin[1]), int(origin[2]), ex, ey, ez, seeds2.ctypes.data,
                                  W.ctypes.data, seeds2.shape[0], m.ctypes.data, out.itemsize, out.ctypes.data)
    return out


def voronoi_device(dims, seeds2, W, metric, weighted: bool, device="cuda"):
    """Same volume as voronoi_host, generated on the GPU (torch tensor)."""
    import torch
    nx, ny, nz = dims
    out = torch.empty((nz, ny, nx), dtype=torch.uint16 if seeds2.shape[0] <= 65536 else torch.int32,
                      device=device)
    s = torch.from_numpy(seeds2).to(device)
    w = torch.from_numpy(W).to(device)
    m = np.ascontiguousarray(np.array(metric, dtype=np.int64))
    stream = torch.cuda.current_stream(out.device).cuda_stream
    rc = _dev_lib().mgs_voronoi_dev(nx, ny, nz, s.data_ptr(), w.data_ptr() if weighted else None,
                                    seeds2.shape[0], m.ctypes.data, out.element_size(),
                                    out.data_ptr(), stream)
    if rc:
        raise RuntimeError("GPU volume generator failed (%d)" % rc)
    torch.cuda.current_stream(out.device).synchronize()
    return out


def cylinders_host(dims, K: int, rng: np.random.Generator, radius=(2.0, 6.0), length=(50.0, 600.0),
                   tries: int = 32):
    """Background 0 plus K non-overlapping cylinders, IDs 1..K (see
    csrc/synth_host.c).  Returns (volume uint16 (z, y, x), background count)."""
    nx, ny, nz = dims
    u = rng.random((K, tries, 8))
    g = rng.standard_normal((K, tries, 3))
    u[:, :, 2:5] = g
    u = np.ascontiguousarray(u)
    vol = np.zeros((nz, ny, nx), dtype=np.uint16)
    bg = _host_lib().mgs_cylinders(nx, ny, nz, K, tries, u.ctypes.data, radius[0], radius[1],
                                   length[0], length[1], vol.ctypes.data)
    return vol, int(bg)


def make_volume(cfg_index: int, device: str = "cpu", dims=None, S=None):
    """The volume of one config (or a resized variant with the same recipe).

    device='cpu' returns a numpy array (z, y, x); device='cuda' a torch tensor
    (Voronoi configs only; cylinder volumes are made on the host)."""
    cfg = CONFIGS[cfg_index]
    dims = tuple(dims) if dims is not None else cfg["dims"]
    S = int(S) if S is not None else cfg["S"]
    rng = rng_for(cfg_index, _STREAM_VOLUME)
    if cfg["kind"] == "voronoi":
        seeds2, W = voronoi_seeds(dims, S, cfg["weighted"], rng)
        if device == "cpu":
            return voronoi_host(dims, seeds2, W, cfg["metric"])
        return voronoi_device(dims, seeds2, W, cfg["metric"], cfg["weighted"], device)
    vol, _ = cylinders_host(dims, S - 1, rng, cfg["radius"], cfg["length"], cfg["tries"])
    if device == "cpu":
        return vol
    import torch
    return torch.from_numpy(vol).to(device)


# --------------------------------------------------------------------------
# boxes, transfer functions, ray samples
# --------------------------------------------------------------------------
def make_boxes(cfg_index: int, Q: int = None, dims=None, box="default", box_max=None,
               stream_offset: int = 0) -> np.ndarray:
    """(Q, 6) int32 boxes (x, y, z, dx, dy, dz), fully inside the volume.

    uniform:    each side uniform in 1..box_max (clamped to the dim)
    loguniform: side = floor(2^U(0, log2(box_max + 1))), clamped to [1, dim]
    The origin is uniform in [0, dim - side]."""
    cfg = CONFIGS[cfg_index]
    dims = tuple(dims) if dims is not None else cfg["dims"]
    Q = int(Q) if Q is not None else cfg["queries"]
    kind = cfg["box"] if box == "default" else box
    bmax = int(box_max) if box_max is not None else cfg["box_max"]
    rng = rng_for(cfg_index, _STREAM_BOXES + 16 * stream_offset)
    d = np.array(dims, dtype=np.int64)
    if kind == "uniform":
        side = rng.integers(1, bmax + 1, size=(Q, 3), dtype=np.int64)
    else:
        u = rng.random((Q, 3))
        side = np.floor(np.exp2(u * math.log2(bmax + 1))).astype(np.int64)
    side = np.clip(side, 1, np.minimum(d, bmax)[None, :])
    origin = np.floor(rng.random((Q, 3)) * (d[None, :] - side + 1)).astype(np.int64)
    origin = np.minimum(origin, d[None, :] - side)
    return np.ascontiguousarray(np.concatenate([origin, side], axis=1).astype(np.int32))


def make_tf(cfg_index: int, S: int, C: int = 4, frame: int = 0) -> np.ndarray:
    """(S, C) float32 transfer function, uniform in [0, 1) per segment."""
    rng = rng_for(cfg_index, _STREAM_TF + 16 * frame)
    return rng.random((S, C), dtype=np.float32)


def make_attribute_tf(cfg_index: int, S: int, frame: int = 0) -> np.ndarray:
    """(S, 4) float32 multi-dimensional TF for the cylinder volume: RGB from a
    random per-segment attribute, opacity = base opacity x |axis . view|."""
    rng = rng_for(cfg_index, _STREAM_TF + 16 * frame)
    rgb = rng.random((S, 3), dtype=np.float32)
    base = rng.random(S, dtype=np.float32)
    g = rng.standard_normal((S, 3))
    g /= np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-12)
    view = rng.standard_normal(3)
    view /= np.linalg.norm(view)
    a = (base * np.abs(g @ view)).astype(np.float32)
    tf = np.concatenate([rgb, a[:, None]], axis=1).astype(np.float32)
    tf[0] = 0.0  # background fully transparent
    return np.ascontiguousarray(tf)


def orbit_camera(cfg_index: int, dims=None, width: int = 1920, height: int = 1080, frame: int = 0,
                 base_step: float = 0.5, lod_bias: int = 0, ert: float = 0.99, max_steps: int = 1 << 20) -> dict:
    """The seeded orbit camera of make_samples as a pinhole camera for the ray
    marcher: eye, orthonormal (fwd, right, up), pixel angle, image size, and
    the march settings (lattice step in level-0 voxels, integer LOD bias,
    early-termination opacity, step cap).  Same draws as make_samples."""
    cfg = CONFIGS[cfg_index]
    dims = np.array(dims if dims is not None else cfg["dims"], dtype=np.float64)
    rng = rng_for(cfg_index, _STREAM_SAMPLES + 16 * frame)
    centre = dims / 2.0
    R = 1.5 * dims.max()
    phi = rng.random() * 2 * math.pi
    eye = centre + R * np.array([math.cos(phi), math.sin(phi), 0.35])
    fwd = centre - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    pix = 2 * math.tan(math.radians(45.0) / 2) / height
    f32 = lambda v: [float(np.float32(x)) for x in v]
    return dict(eye=f32(eye), fwd=f32(fwd), right=f32(right), up=f32(up), pix=float(np.float32(pix)),
                width=int(width), height=int(height), base_step=float(base_step), lod_bias=int(lod_bias),
                ert=float(ert), max_steps=int(max_steps))


def make_samples(cfg_index: int, dims=None, width: int = 1920, height: int = 1080, frame: int = 0,
                 lod_bias: float = 0.0) -> np.ndarray:
    """(width*height, 4) float32 ray samples (x, y, z, lod) for one frame.

    An orbit camera circles the volume at 1.5x its largest extent with a 45
    degree vertical field of view; each pixel's sample lies at a uniform depth
    inside the ray's intersection with the volume, and its LOD is
    log2(t * pixel_angle) + bias (pixel footprint linear in depth, Sec. 4)."""
    cfg = CONFIGS[cfg_index]
    dims = np.array(dims if dims is not None else cfg["dims"], dtype=np.float64)
    rng = rng_for(cfg_index, _STREAM_SAMPLES + 16 * frame)
    centre = dims / 2.0
    R = 1.5 * dims.max()
    phi = rng.random() * 2 * math.pi
    eye = centre + R * np.array([math.cos(phi), math.sin(phi), 0.35])
    fwd = centre - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    fov = math.radians(45.0)
    pix = 2 * math.tan(fov / 2) / height
    jj, ii = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    sx = (ii + 0.5 - width / 2) * pix
    sy = (height / 2 - jj - 0.5) * pix
    dirs = fwd[None, None, :] + sx[..., None] * right[None, None, :] + sy[..., None] * up[None, None, :]
    dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
    inv = 1.0 / np.where(np.abs(dirs) < 1e-12, 1e-12, dirs)
    t0 = (0.0 - eye) * inv
    t1 = (dims - eye) * inv
    tmin = np.minimum(t0, t1).max(axis=-1)
    tmax = np.maximum(t0, t1).min(axis=-1)
    hit = tmax > np.maximum(tmin, 0.0)
    tmin = np.maximum(tmin, 0.0)
    tc = np.linalg.norm(centre - eye)
    tmin = np.where(hit, tmin, tc)
    tmax = np.where(hit, tmax, tc)
    t = tmin + rng.random((height, width)) * (tmax - tmin)
    pos = eye[None, None, :] + t[..., None] * dirs
    lod = np.log2(np.maximum(t * pix, 1e-30)) + lod_bias
    out = np.concatenate([pos, lod[..., None]], axis=-1).reshape(-1, 4).astype(np.float32)
    return np.ascontiguousarray(out)


# --------------------------------------------------------------------------
# request streams for the serving loop
# --------------------------------------------------------------------------
def make_request_mix(n: int, rate: float, vol_dims, box_max, tf_frac: float = 0.1, stream_offset: int = 0,
                     cfg_index: int = 5):
    """A Poisson request stream over several volumes.

    Returns (arrival seconds (n,), kind (n,) 0 = box / 1 = TF frame,
    volume (n,), boxes (n, 6) int32).  Inter-arrival gaps are exponential with
    mean 1/rate; each request picks a volume uniformly and is a TF frame with
    probability tf_frac; box sides are floor(2^U(0, log2(box_max[v] + 1)))
    clamped to the volume (vol_dims[v] = (nx, ny, nz)), origins uniform so the
    box lies inside.  Boxes of TF frames are unused (zero)."""
    rng = rng_for(cfg_index, _STREAM_BOXES + 16 * stream_offset)
    gaps = rng.exponential(1.0 / rate, size=n)
    arrival = np.cumsum(gaps) - gaps[0]
    kind = (rng.random(n) < tf_frac).astype(np.int32)
    volume = rng.integers(0, len(vol_dims), size=n).astype(np.int32)
    boxes = np.zeros((n, 6), np.int32)
    u = rng.random((n, 3))
    o = rng.random((n, 3))
    for v, dims in enumerate(vol_dims):
        m = (volume == v) & (kind == 0)
        d = np.array(dims, dtype=np.int64)
        bm = int(box_max[v])
        side = np.floor(np.exp2(u[m] * math.log2(bm + 1))).astype(np.int64)
        side = np.clip(side, 1, np.minimum(d, bm)[None, :])
        origin = np.minimum(np.floor(o[m] * (d[None, :] - side + 1)).astype(np.int64), d[None, :] - side)
        boxes[m] = np.concatenate([origin, side], axis=1).astype(np.int32)
    return arrival, kind, volume, boxes
