"""Thin Python binding of libmg (the C-ABI declared in include/mg.h).

Each function carries the name of the C entry point it marshals arguments
for; all computation happens in the library's CUDA kernels.  PyTorch supplies
device memory (tensors, and the caching allocator behind the library's
allocator callback) and streams.  There is no fallback: if the compiled
library is missing, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmg.so")

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_OOM, MG_ERR_CUDA = 0, 1, 2, 3
MG_ERR_TIMEOUT, MG_ERR_CAPACITY, MG_ERR_UNSUPPORTED, MG_ERR_INEXACT = 4, 5, 6, 7
MG_ERR_CANCELLED = 8
MG_REQ_BOX, MG_REQ_TF = 0, 1
MG_F32, MG_F16, MG_BF16 = 0, 1, 2
MG_HIST_U32, MG_HIST_F32 = 0, 1
MG_LAYOUT_DENSE, MG_LAYOUT_CSR = 0, 1
MG_SCHED_BATCHED, MG_SCHED_PLAIN, MG_SCHED_NAIVE = 0, 1, 2
_SCHED = {"batched": MG_SCHED_BATCHED, "plain": MG_SCHED_PLAIN, "naive": MG_SCHED_NAIVE}
MG_MAX_LEVELS, MG_MAX_DEPTH = 32, 64
MG_NO_NODE = 0xFFFFFFFF

_DTYPES = {"f32": (MG_F32, torch.float32), "f16": (MG_F16, torch.float16), "bf16": (MG_BF16, torch.bfloat16)}
_TORCH_TO_MG = {torch.float32: MG_F32, torch.float16: MG_F16, torch.bfloat16: MG_BF16}

# names of every symbol include/mg.h declares (checked by the CPU tests)
EXPORTS = ("mg_build", "mg_graph_info_get", "mg_graph_copy_nodes", "mg_graph_copy_mip", "mg_propagate_tf",
           "mg_query_boxes", "mg_query_boxes_noalloc", "mg_query_timing",
           "mg_query_plan_create", "mg_query_plan_run", "mg_query_plan_timing", "mg_query_plan_free",
           "mg_query_autotune",
           "mg_query_set_tuning", "mg_count_cubes", "mg_render_lookup", "mg_propagate_tf_multi",
           "mg_render_lookup_multi", "mg_raymarch", "mg_bitstream_size", "mg_bitstream_write", "mg_bitstream_parse",
           "mg_bitstream_decode_mip", "mg_bitstream_decode_nodes", "mg_bitstream_lookup",
           "mg_factor_greedy", "mg_greedy_info_get", "mg_greedy_copy_nodes", "mg_greedy_copy_mip",
           "mg_greedy_copy_picks", "mg_greedy_copy_codebook", "mg_greedy_free", "mg_graph_from_greedy",
           "mg_error_table_build", "mg_error_table_copy", "mg_query_lut",
           "mg_server_create", "mg_server_add_volume", "mg_server_remove_volume", "mg_server_start", "mg_server_submit", "mg_server_cancel",
           "mg_server_wait", "mg_server_replay", "mg_server_stats_get", "mg_server_free",
           "mg_graph_export_size", "mg_graph_export", "mg_graph_import",
           "mg_selftest_bounded_wait", "mg_sync_status", "mg_free", "mg_last_error", "mg_version")


class MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("mg status %d: %s" % (status, msg))
        self.status = status


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class mg_allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class mg_build_opts(ctypes.Structure):
    _fields_ = [("id_bytes", ctypes.c_int), ("reserved", ctypes.c_int * 7)]


class mg_graph_info(ctypes.Structure):
    _fields_ = [("num_segments", ctypes.c_uint32), ("levels", ctypes.c_int), ("depth", ctypes.c_int),
                ("num_nodes", ctypes.c_int64), ("dims", (ctypes.c_int64 * 3) * MG_MAX_LEVELS),
                ("bucket", ctypes.c_int64 * (MG_MAX_DEPTH + 2)), ("max_list", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("build_ms", ctypes.c_double),
                ("lut_entries", ctypes.c_int64)]


class mg_query_opts(ctypes.Structure):
    _fields_ = [("hist_type", ctypes.c_int), ("layout", ctypes.c_int), ("alpha_dtype", ctypes.c_int),
                ("schedule", ctypes.c_int), ("chunk_cubes", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("timing", ctypes.c_int), ("reserved", ctypes.c_int)]


class mg_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("pix", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("base_step", ctypes.c_float), ("lod_bias", ctypes.c_int32),
                ("ert", ctypes.c_float), ("max_steps", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


def camera(cam: dict) -> mg_camera:
    """mg_camera from a dict (eye, fwd, right, up, pix, width, height,
    base_step, lod_bias, ert, max_steps), e.g. synth.orbit_camera()."""
    c = mg_camera()
    for k in ("eye", "fwd", "right", "up"):
        for i in range(3):
            getattr(c, k)[i] = float(cam[k][i])
    c.pix, c.width, c.height = float(cam["pix"]), int(cam["width"]), int(cam["height"])
    c.base_step, c.lod_bias, c.ert, c.max_steps = float(cam["base_step"]), int(cam["lod_bias"]), float(cam["ert"]), \
        int(cam["max_steps"])
    return c


class mg_bitstream_info(ctypes.Structure):
    _fields_ = [("num_segments", ctypes.c_uint32), ("levels", ctypes.c_int), ("node_bits", ctypes.c_int),
                ("weight_bits", ctypes.c_int), ("num_nodes", ctypes.c_int64),
                ("dims", (ctypes.c_int64 * 3) * MG_MAX_LEVELS), ("voxel_bits", ctypes.c_int32 * MG_MAX_LEVELS),
                ("imin", ctypes.c_int64 * MG_MAX_LEVELS), ("level_bit", ctypes.c_int64 * MG_MAX_LEVELS),
                ("node_bit", ctypes.c_int64), ("header_bits", ctypes.c_int64), ("bytes", ctypes.c_int64)]


class mg_greedy_opts(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int), ("tau", ctypes.c_int), ("bitrate", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class mg_greedy_info(ctypes.Structure):
    _fields_ = [("num_segments", ctypes.c_uint32), ("levels", ctypes.c_int), ("depth", ctypes.c_int),
                ("reserved0", ctypes.c_int), ("num_nodes", ctypes.c_int64), ("picks", ctypes.c_int64),
                ("waves", ctypes.c_int64), ("ms", ctypes.c_double)]


class mg_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_batch", ctypes.c_int), ("hist_type", ctypes.c_int),
                ("storage", ctypes.c_int), ("max_samples", ctypes.c_int64), ("memory_budget", ctypes.c_int64),
                ("plain", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class mg_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("volume", ctypes.c_int), ("box", ctypes.c_int32 * 6),
                ("tf", ctypes.c_void_p), ("samples", ctypes.c_void_p), ("P", ctypes.c_int64),
                ("result", ctypes.c_void_p), ("arrival_s", ctypes.c_double)]


class mg_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("box_requests", "tf_requests", "box_launches", "max_batch_seen",
                                              "cancelled", "failed", "memory_admitted", "tf_launches")]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libmg.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmg.so is not built (%s): run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int
        L.mg_build.argtypes = [P, i64, i64, i64, ctypes.c_uint32, ctypes.POINTER(mg_build_opts),
                               ctypes.POINTER(mg_allocator), P, ctypes.POINTER(P)]
        L.mg_build.restype = st
        L.mg_graph_info_get.argtypes = [P, ctypes.POINTER(mg_graph_info)]
        L.mg_graph_info_get.restype = st
        L.mg_graph_copy_nodes.argtypes = [P, P, P, P, P, P]
        L.mg_graph_copy_nodes.restype = st
        L.mg_graph_copy_mip.argtypes = [P, i32, P, P]
        L.mg_graph_copy_mip.restype = st
        L.mg_propagate_tf.argtypes = [P, P, i32, i32, P, P]
        L.mg_propagate_tf.restype = st
        L.mg_propagate_tf_multi.argtypes = [P, P, i32, i32, i32, P, P]
        L.mg_propagate_tf_multi.restype = st
        L.mg_render_lookup_multi.argtypes = [P, P, i32, i32, i32, P, P, P, P]
        L.mg_render_lookup_multi.restype = st
        L.mg_raymarch.argtypes = [P, P, P, ctypes.POINTER(mg_camera), P, P, P]
        L.mg_factor_greedy.argtypes = [P, i64, i64, i64, ctypes.c_uint32, ctypes.POINTER(mg_build_opts),
                                       ctypes.POINTER(mg_greedy_opts), P, ctypes.POINTER(P)]
        L.mg_greedy_info_get.argtypes = [P, ctypes.POINTER(mg_greedy_info)]
        L.mg_greedy_copy_nodes.argtypes = [P, P, P, P, P]
        L.mg_greedy_copy_mip.argtypes = [P, i32, P]
        L.mg_greedy_copy_picks.argtypes = [P, P]
        L.mg_greedy_copy_codebook.argtypes = [P, P, P]
        for f in ("mg_factor_greedy", "mg_greedy_info_get", "mg_greedy_copy_nodes", "mg_greedy_copy_mip",
                  "mg_greedy_copy_picks", "mg_greedy_copy_codebook"):
            getattr(L, f).restype = st
        L.mg_graph_from_greedy.argtypes = [P, ctypes.POINTER(mg_allocator), P, ctypes.POINTER(P)]
        L.mg_graph_from_greedy.restype = st
        L.mg_error_table_build.argtypes = [P, ctypes.POINTER(ctypes.c_int64), P]
        L.mg_error_table_build.restype = st
        L.mg_error_table_copy.argtypes = [P, P, P, P, P]
        L.mg_error_table_copy.restype = st
        L.mg_query_lut.argtypes = [P, P, i64, P, P, P]
        L.mg_query_lut.restype = st
        L.mg_greedy_free.argtypes = [P]
        L.mg_greedy_free.restype = None
        L.mg_bitstream_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.mg_bitstream_write.argtypes = [P, P, ctypes.c_size_t, P]
        L.mg_bitstream_parse.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(mg_bitstream_info)]
        L.mg_bitstream_decode_mip.argtypes = [P, ctypes.POINTER(mg_bitstream_info), i32, P, P]
        L.mg_bitstream_decode_nodes.argtypes = [P, ctypes.POINTER(mg_bitstream_info), P, P, P, P, P]
        L.mg_bitstream_lookup.argtypes = [P, ctypes.POINTER(mg_bitstream_info), P, i32, i32, P, i64, P, P]
        for f in ("mg_bitstream_size", "mg_bitstream_write", "mg_bitstream_parse", "mg_bitstream_decode_mip",
                  "mg_bitstream_decode_nodes", "mg_bitstream_lookup"):
            getattr(L, f).restype = st
        L.mg_raymarch.restype = st
        L.mg_query_boxes.argtypes = [P, P, i64, ctypes.POINTER(mg_query_opts), P, ctypes.c_size_t, P, P,
                                     ctypes.POINTER(ctypes.c_size_t), P]
        L.mg_query_boxes.restype = st
        L.mg_query_boxes_noalloc.argtypes = [P, P, i64, P, ctypes.c_size_t, P]
        L.mg_query_boxes_noalloc.restype = st
        L.mg_query_plan_create.argtypes = [P, i64, ctypes.POINTER(mg_query_opts), i64, i64, ctypes.POINTER(P)]
        L.mg_query_plan_create.restype = st
        L.mg_query_plan_run.argtypes = [P, P, i64, P, ctypes.c_size_t, P]
        L.mg_query_plan_run.restype = st
        L.mg_query_plan_timing.argtypes = [P, P, P]
        L.mg_query_plan_timing.restype = st
        L.mg_query_plan_free.argtypes = [P]
        L.mg_query_plan_free.restype = None
        L.mg_query_autotune.argtypes = [P, P, i64, ctypes.POINTER(mg_query_opts), ctypes.POINTER(ctypes.c_float), P]
        L.mg_query_autotune.restype = st
        L.mg_query_set_tuning.argtypes = [P, i32, i32, i32]
        L.mg_query_set_tuning.restype = st
        L.mg_query_timing.argtypes = [P, P, P, P]
        L.mg_query_timing.restype = st
        L.mg_count_cubes.argtypes = [P, P, i64, P, P]
        L.mg_count_cubes.restype = st
        L.mg_render_lookup.argtypes = [P, P, i32, i32, P, i64, P, P]
        L.mg_render_lookup.restype = st
        L.mg_server_create.argtypes = [ctypes.POINTER(mg_server_opts), ctypes.POINTER(P)]
        L.mg_server_create.restype = st
        L.mg_server_add_volume.argtypes = [P, P, i32, ctypes.POINTER(ctypes.c_int)]
        L.mg_server_add_volume.restype = st
        L.mg_server_remove_volume.argtypes = [P, i32, ctypes.c_double]
        L.mg_server_remove_volume.restype = st
        L.mg_server_start.argtypes = [P]
        L.mg_server_start.restype = st
        L.mg_server_submit.argtypes = [P, ctypes.POINTER(mg_request), ctypes.POINTER(ctypes.c_uint64)]
        L.mg_server_submit.restype = st
        L.mg_server_cancel.argtypes = [P, ctypes.c_uint64]
        L.mg_server_cancel.restype = st
        L.mg_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        L.mg_server_wait.restype = st
        L.mg_server_replay.argtypes = [P, ctypes.POINTER(mg_request), i64, P, ctypes.POINTER(ctypes.c_double)]
        L.mg_server_replay.restype = st
        L.mg_server_stats_get.argtypes = [P, ctypes.POINTER(mg_server_stats)]
        L.mg_server_stats_get.restype = st
        L.mg_server_free.argtypes = [P]
        L.mg_server_free.restype = None
        L.mg_graph_export_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.mg_graph_export_size.restype = st
        L.mg_graph_export.argtypes = [P, P, ctypes.c_size_t, P]
        L.mg_graph_export.restype = st
        L.mg_graph_import.argtypes = [P, ctypes.c_size_t, ctypes.POINTER(mg_allocator), P, ctypes.POINTER(P)]
        L.mg_graph_import.restype = st
        L.mg_selftest_bounded_wait.argtypes = [i32, ctypes.c_uint, P]
        L.mg_selftest_bounded_wait.restype = st
        L.mg_sync_status.argtypes = [P, P]
        L.mg_sync_status.restype = st
        L.mg_free.argtypes = [P]
        L.mg_free.restype = None
        L.mg_last_error.argtypes = []
        L.mg_last_error.restype = ctypes.c_char_p
        L.mg_version.argtypes = []
        L.mg_version.restype = ctypes.c_char_p
        _lib = L
        return L


def mg_last_error() -> str:
    return lib().mg_last_error().decode()


def mg_version() -> str:
    return lib().mg_version().decode()


def _check(st: int):
    if st != MG_OK:
        raise MGError(st, mg_last_error())


def _stream(stream=None) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


# --------------------------------------------------------------------------
# allocator callback backed by torch's caching allocator
# --------------------------------------------------------------------------
def _torch_alloc(ctx, nbytes, stream):
    try:
        dev = int(ctx or 0)
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
    except Exception:
        return None


def _torch_free(ctx, ptr, nbytes, stream):
    try:
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


_ALLOC_CB = ALLOC_FN(_torch_alloc)
_FREE_CB = FREE_FN(_torch_free)


def torch_allocator(device: int) -> mg_allocator:
    return mg_allocator(ctypes.c_void_p(device), _ALLOC_CB, _FREE_CB)


# --------------------------------------------------------------------------
# entry points
# --------------------------------------------------------------------------
class Graph:
    """Owns an mg_graph handle (released by mg_free)."""

    def __init__(self, handle: int, device: int, allocator):
        self.handle = handle
        self.device = device
        self._allocator = allocator   # keeps the callback struct alive
        self.info = mg_graph_info_get(self)

    @property
    def S(self):
        return self.info["num_segments"]

    @property
    def N(self):
        return self.info["num_nodes"]

    def close(self):
        if self.handle:
            mg_free(self)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_build(ids: torch.Tensor, num_segments: int, stream=None, use_torch_allocator: bool = True) -> Graph:
    """Build the Mixture Graph of a (nz, ny, nx) uint16/uint32/int32 ID volume on the GPU."""
    if not ids.is_cuda or ids.dim() != 3:
        raise ValueError("ids must be a 3-D CUDA tensor (z, y, x)")
    ids = ids.contiguous()
    if ids.dtype == torch.uint16:
        nb = 2
    elif ids.dtype in (torch.uint32, torch.int32):
        nb = 4
    else:
        raise TypeError("ids must be uint16, uint32 or int32")
    nz, ny, nx = ids.shape
    opts = mg_build_opts(nb)
    dev = ids.device.index if ids.device.index is not None else torch.cuda.current_device()
    alloc = torch_allocator(dev) if use_torch_allocator else None
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        st = lib().mg_build(ids.data_ptr(), nx, ny, nz, num_segments, ctypes.byref(opts),
                            ctypes.byref(alloc) if alloc is not None else None, _stream(stream),
                            ctypes.byref(h))
    _check(st)
    return Graph(h.value, dev, alloc)


def mg_graph_info_get(g: Graph) -> dict:
    info = mg_graph_info()
    _check(lib().mg_graph_info_get(g.handle, ctypes.byref(info)))
    L, D = info.levels, info.depth
    return dict(num_segments=info.num_segments, levels=L, depth=D, num_nodes=info.num_nodes,
                dims=[tuple(info.dims[l][k] for k in range(3)) for l in range(L)],
                bucket=[info.bucket[d] for d in range(D + 2)], max_list=info.max_list, pairs=info.pairs,
                device_bytes=info.device_bytes, build_ms=info.build_ms, lut_entries=info.lut_entries)


def mg_graph_copy_nodes(g: Graph, stream=None):
    """(p, q, a, b) numpy arrays of the canonical node table."""
    import numpy as np
    N = g.N
    p = np.zeros(N, np.uint32); q = np.zeros(N, np.uint32)
    a = np.zeros(N, np.uint64); b = np.zeros(N, np.uint64)
    _check(lib().mg_graph_copy_nodes(g.handle, p.ctypes.data, q.ctypes.data, a.ctypes.data, b.ctypes.data,
                                     _stream(stream)))
    return p, q, a, b


def mg_graph_copy_mip(g: Graph, level: int, stream=None):
    """Node IDs of one level, numpy uint32 array (z, y, x)."""
    import numpy as np
    nx, ny, nz = g.info["dims"][level]
    out = np.zeros((nz, ny, nx), np.uint32)
    _check(lib().mg_graph_copy_mip(g.handle, level, out.ctypes.data, _stream(stream)))
    return out


def _check_out(out, shape, dtype, device, name="out"):
    """A caller's output tensor is written through its data pointer: it must be
    contiguous, with the shape, dtype and device of the result."""
    if (not isinstance(out, torch.Tensor) or out.dtype != dtype or tuple(out.shape) != tuple(shape)
            or out.device != device or not out.is_contiguous()):
        raise ValueError("%s must be a contiguous %s tensor of shape %s on %s" % (name, dtype, tuple(shape), device))
    return out


def mg_propagate_tf(g: Graph, tf: torch.Tensor, storage: str = "f32", out: torch.Tensor = None,
                    stream=None) -> torch.Tensor:
    """Node values (N, C) in `storage` dtype from an (S, C) fp32 CUDA transfer function."""
    if not tf.is_cuda or tf.dtype != torch.float32 or tf.dim() != 2 or tf.shape[0] != g.S:
        raise ValueError("tf must be a CUDA float32 tensor of shape (S, C)")
    tf = tf.contiguous()
    code, dt = _DTYPES[storage]
    C = tf.shape[1]
    if out is None:
        out = torch.empty((g.N, C), dtype=dt, device=tf.device)
    _check_out(out, (g.N, C), dt, tf.device)
    _check(lib().mg_propagate_tf(g.handle, tf.data_ptr(), C, code, out.data_ptr(), _stream(stream)))
    return out


def mg_propagate_tf_multi(g: Graph, tfs: torch.Tensor, storage: str = "f32", out: torch.Tensor = None,
                          stream=None) -> torch.Tensor:
    """Node values (N, k*C) of k transfer functions (k, S, C) fp32 in one pass;
    columns [j*C, (j+1)*C) hold TF j's values."""
    if not tfs.is_cuda or tfs.dtype != torch.float32 or tfs.dim() != 3 or tfs.shape[1] != g.S:
        raise ValueError("tfs must be a CUDA float32 tensor of shape (k, S, C)")
    tfs = tfs.contiguous()
    code, dt = _DTYPES[storage]
    k, C = tfs.shape[0], tfs.shape[2]
    if out is None:
        out = torch.empty((g.N, k * C), dtype=dt, device=tfs.device)
    _check_out(out, (g.N, k * C), dt, tfs.device)
    _check(lib().mg_propagate_tf_multi(g.handle, tfs.data_ptr(), k, C, code, out.data_ptr(), _stream(stream)))
    return out


def mg_render_lookup_multi(g: Graph, vals: torch.Tensor, k: int, samples: torch.Tensor, offsets,
                           out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """Lookups of k frames: samples (P, 4), offsets (k+1,) host ints; frame j's
    samples read columns [j*C, (j+1)*C) of vals (N, k*C).  Returns (P, C)."""
    import numpy as np
    if samples.dtype != torch.float32 or samples.dim() != 2 or samples.shape[1] != 4:
        raise ValueError("samples must be float32 of shape (P, 4)")
    if vals.dim() != 2 or vals.shape[1] % k:
        raise ValueError("vals must have k*C columns")
    samples = samples.contiguous()
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off.shape != (k + 1,) or off[-1] != samples.shape[0]:
        raise ValueError("offsets must have k+1 entries ending at the number of samples")
    C = vals.shape[1] // k
    if out is None:
        out = torch.empty((samples.shape[0], C), dtype=vals.dtype, device=vals.device)
    _check_out(out, (samples.shape[0], C), vals.dtype, vals.device)
    _check(lib().mg_render_lookup_multi(g.handle, vals.data_ptr(), k, C, _TORCH_TO_MG[vals.dtype], samples.data_ptr(),
                                        off.ctypes.data, out.data_ptr(), _stream(stream)))
    return out


def mg_query_boxes(g: Graph, boxes: torch.Tensor, hist: str = "u32", layout: str = "dense",
                   alpha: str = "f32", schedule: str = "batched", chunk_cubes: int = 0,
                   block_threads: int = 0, out=None, capacity: int = None, timing: bool = False,
                   stream=None):
    """Segment histograms of (Q, 6) int32 boxes.

    dense: returns a (Q, S) uint32 (hist='u32') or float32 tensor.
    csr:   returns (offsets uint64 (Q+1), seg uint32 (nnz), values (nnz))."""
    if not boxes.is_cuda or boxes.dtype != torch.int32 or boxes.dim() != 2 or boxes.shape[1] != 6:
        raise ValueError("boxes must be a CUDA int32 tensor of shape (Q, 6)")
    boxes = boxes.contiguous()
    Q = boxes.shape[0]
    o = mg_query_opts()
    o.hist_type = MG_HIST_F32 if hist == "f32" else MG_HIST_U32
    o.layout = MG_LAYOUT_CSR if layout == "csr" else MG_LAYOUT_DENSE
    o.alpha_dtype = _DTYPES[alpha][0]
    o.schedule = _SCHED[schedule]
    o.chunk_cubes = chunk_cubes
    o.block_threads = block_threads
    o.timing = 1 if timing else 0
    vdt = torch.float32 if hist == "f32" else torch.uint32
    req = ctypes.c_size_t(0)
    dev = boxes.device
    if layout != "csr":
        if out is None:
            out = torch.empty((Q, g.S), dtype=vdt, device=dev)
        _check_out(out, (Q, g.S), vdt, dev)
        _check(lib().mg_query_boxes(g.handle, boxes.data_ptr(), Q, ctypes.byref(o), out.data_ptr(),
                                    out.numel(), None, None, ctypes.byref(req), _stream(stream)))
        return out
    offsets = torch.empty(Q + 1, dtype=torch.uint64, device=dev)
    cap = int(capacity) if capacity is not None else 0
    for _ in range(2):
        seg = torch.empty(max(cap, 1), dtype=torch.uint32, device=dev)
        vals = torch.empty(max(cap, 1), dtype=vdt, device=dev)
        st = lib().mg_query_boxes(g.handle, boxes.data_ptr(), Q, ctypes.byref(o), vals.data_ptr(), cap,
                                  seg.data_ptr(), offsets.data_ptr(), ctypes.byref(req), _stream(stream))
        if st == MG_ERR_CAPACITY and capacity is None:
            cap = int(req.value)
            continue
        _check(st)
        n = int(req.value)
        return offsets, seg[:n], vals[:n]
    raise MGError(MG_ERR_CAPACITY, mg_last_error())


def mg_query_boxes_noalloc(g: Graph, boxes: torch.Tensor, out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """Exact dense (Q, S) uint32 histograms with the library's fixed scratch:
    for callers that must not allocate device memory (the output is theirs)."""
    if not boxes.is_cuda or boxes.dtype != torch.int32 or boxes.dim() != 2 or boxes.shape[1] != 6:
        raise ValueError("boxes must be a CUDA int32 tensor of shape (Q, 6)")
    boxes = boxes.contiguous()
    Q = boxes.shape[0]
    if out is None:
        out = torch.empty((Q, g.S), dtype=torch.uint32, device=boxes.device)
    _check_out(out, (Q, g.S), torch.uint32, boxes.device)
    _check(lib().mg_query_boxes_noalloc(g.handle, boxes.data_ptr(), Q, out.data_ptr(), out.numel(),
                                        _stream(stream)))
    return out


class QueryPlan:
    """A captured batched query (mg_query_plan_*): one graph launch per batch."""

    def __init__(self, g: Graph, max_Q: int, hist: str = "u32", alpha: str = "f32", chunk_cubes: int = 0,
                 block_threads: int = 0, max_blocks: int = 0, max_chunks: int = 0, timing: bool = False):
        o = mg_query_opts()
        o.hist_type = MG_HIST_F32 if hist == "f32" else MG_HIST_U32
        o.alpha_dtype = _DTYPES[alpha][0]
        o.chunk_cubes = chunk_cubes
        o.block_threads = block_threads
        o.timing = 1 if timing else 0
        h = ctypes.c_void_p()
        with torch.cuda.device(g.device):
            _check(lib().mg_query_plan_create(g.handle, max_Q, ctypes.byref(o), max_blocks, max_chunks,
                                              ctypes.byref(h)))
        self.handle = h.value
        self.graph = g
        self.max_Q = max_Q
        self.dtype = torch.float32 if hist == "f32" else torch.uint32

    def run(self, boxes: torch.Tensor, out: torch.Tensor = None, stream=None) -> torch.Tensor:
        """mg_query_plan_run: (Q, S) histograms of (Q, 6) int32 CUDA boxes."""
        boxes = boxes.contiguous()
        Q = boxes.shape[0]
        if out is None:
            out = torch.empty((Q, self.graph.S), dtype=self.dtype, device=boxes.device)
        _check_out(out, (Q, self.graph.S), self.dtype, boxes.device)
        _check(lib().mg_query_plan_run(self.handle, boxes.data_ptr(), Q, out.data_ptr(), out.numel(),
                                       _stream(stream)))
        return out

    def timing(self):
        """(plan_ms, main_ms) of the last run (plans created with timing=True)."""
        t = [ctypes.c_float(), ctypes.c_float()]
        _check(lib().mg_query_plan_timing(self.handle, *[ctypes.byref(x) for x in t]))
        return tuple(x.value for x in t)

    def close(self):
        if self.handle:
            lib().mg_query_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_query_plan_create(g: Graph, max_Q: int, **kw) -> QueryPlan:
    return QueryPlan(g, max_Q, **kw)


def mg_query_autotune(g: Graph, boxes: torch.Tensor, hist: str = "u32", alpha: str = "f32", cache: str = None,
                      key: str = None, stream=None) -> dict:
    """Choose the batched query's launch shape on this batch and keep it in the
    graph.  With `cache` (a JSON file) and `key`, a shape found before under
    the same GPU name and key is reused without timing."""
    import json
    dev = torch.cuda.get_device_name(g.device)
    full_key = "%s|%s|%s" % (dev, key, hist) if key else None
    ht = MG_HIST_F32 if hist == "f32" else MG_HIST_U32
    if cache and full_key and os.path.exists(cache):
        try:
            with open(cache) as f:
                hit = json.load(f).get(full_key)
        except (OSError, ValueError):
            hit = None
        if hit:
            _check(lib().mg_query_set_tuning(g.handle, ht, int(hit["chunk_cubes"]), int(hit["block_threads"])))
            return dict(hit, cached=True)
    boxes = boxes.contiguous()
    o = mg_query_opts()
    o.hist_type = ht
    o.alpha_dtype = _DTYPES[alpha][0]
    best = ctypes.c_float(0)
    _check(lib().mg_query_autotune(g.handle, boxes.data_ptr(), boxes.shape[0], ctypes.byref(o), ctypes.byref(best),
                                   _stream(stream)))
    res = {"chunk_cubes": o.chunk_cubes, "block_threads": o.block_threads, "best_ms": best.value}
    if cache and full_key:
        data = {}
        try:
            with open(cache) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
        data[full_key] = res
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        tmp = cache + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return dict(res, cached=False)


def mg_query_timing(g: Graph):
    """(plan_ms, main_ms, output_ms) of the last query call made with timing=True."""
    t = [ctypes.c_float(), ctypes.c_float(), ctypes.c_float()]
    _check(lib().mg_query_timing(g.handle, *[ctypes.byref(x) for x in t]))
    return tuple(x.value for x in t)


def mg_count_cubes(g: Graph, boxes: torch.Tensor, stream=None) -> torch.Tensor:
    """Footprint-assembly cube (fetch) count per box, uint64 (Q,)."""
    boxes = boxes.contiguous()
    out = torch.empty(boxes.shape[0], dtype=torch.uint64, device=boxes.device)
    _check(lib().mg_count_cubes(g.handle, boxes.data_ptr(), boxes.shape[0], out.data_ptr(), _stream(stream)))
    return out


def mg_render_lookup(g: Graph, vals: torch.Tensor, samples: torch.Tensor, out: torch.Tensor = None,
                     stream=None) -> torch.Tensor:
    """Value row of the node under every (x, y, z, lod) sample, (P, C) in vals' dtype."""
    if samples.dtype != torch.float32 or samples.dim() != 2 or samples.shape[1] != 4:
        raise ValueError("samples must be float32 of shape (P, 4)")
    samples = samples.contiguous()
    C = vals.shape[1]
    if out is None:
        out = torch.empty((samples.shape[0], C), dtype=vals.dtype, device=vals.device)
    _check_out(out, (samples.shape[0], C), vals.dtype, vals.device)
    _check(lib().mg_render_lookup(g.handle, vals.data_ptr(), C, _TORCH_TO_MG[vals.dtype], samples.data_ptr(),
                                  samples.shape[0], out.data_ptr(), _stream(stream)))
    return out


def mg_raymarch(g: Graph, vals: torch.Tensor, cam: dict, opacity: torch.Tensor = None, image: torch.Tensor = None,
                steps: bool = False, stream=None):
    """RGBA image (H, W, 4) fp32 ray-marched through node values vals (N, 4)
    fp32; with opacity (N,) fp32 empty space is skipped.  steps=True also
    returns the samples composited per pixel (H, W) int32."""
    if vals.dtype != torch.float32 or tuple(vals.shape) != (g.N, 4) or not vals.is_contiguous():
        raise ValueError("vals must be a contiguous float32 tensor of shape (N, 4)")
    if opacity is not None and (opacity.dtype != torch.float32 or tuple(opacity.shape) != (g.N,)
                                or not opacity.is_contiguous()):
        raise ValueError("opacity must be a contiguous float32 tensor of shape (N,)")
    c = camera(cam)
    if image is None:
        image = torch.empty((c.height, c.width, 4), dtype=torch.float32, device=vals.device)
    _check_out(image, (c.height, c.width, 4), torch.float32, vals.device, "image")
    st = torch.empty((c.height, c.width), dtype=torch.int32, device=vals.device) if steps else None
    _check(lib().mg_raymarch(g.handle, vals.data_ptr(), opacity.data_ptr() if opacity is not None else None,
                             ctypes.byref(c), image.data_ptr(), st.data_ptr() if st is not None else None,
                             _stream(stream)))
    return (image, st) if steps else image


class Bitstream:
    """A graph's bitstream (Table 1) in device memory with its parsed layout."""

    def __init__(self, data: torch.Tensor):
        self.data = data
        head = data[:1024].cpu().numpy()
        self.info = mg_bitstream_info()
        _check(lib().mg_bitstream_parse(head.ctypes.data, head.nbytes, ctypes.byref(self.info)))

    def decode_mip(self, level: int, stream=None) -> torch.Tensor:
        """Node IDs of one level, (z, y, x) uint32, decoded on the device."""
        d = self.info.dims[level]
        out = torch.empty((d[2], d[1], d[0]), dtype=torch.uint32, device=self.data.device)
        _check(lib().mg_bitstream_decode_mip(self.data.data_ptr(), ctypes.byref(self.info), level, out.data_ptr(),
                                             _stream(stream)))
        return out

    def decode_nodes(self, stream=None):
        """(p, q, a, b) device tensors of the node table."""
        N, dev = self.info.num_nodes, self.data.device
        p = torch.empty(N, dtype=torch.uint32, device=dev)
        q = torch.empty(N, dtype=torch.uint32, device=dev)
        a = torch.empty(N, dtype=torch.uint64, device=dev)
        b = torch.empty(N, dtype=torch.uint64, device=dev)
        _check(lib().mg_bitstream_decode_nodes(self.data.data_ptr(), ctypes.byref(self.info), p.data_ptr(),
                                               q.data_ptr(), a.data_ptr(), b.data_ptr(), _stream(stream)))
        return p, q, a, b

    def lookup(self, vals: torch.Tensor, samples: torch.Tensor, stream=None) -> torch.Tensor:
        """mg_render_lookup with node IDs read from the stream by bit address."""
        samples = samples.contiguous()
        C = vals.shape[1]
        out = torch.empty((samples.shape[0], C), dtype=vals.dtype, device=vals.device)
        _check(lib().mg_bitstream_lookup(self.data.data_ptr(), ctypes.byref(self.info), vals.data_ptr(), C,
                                         _TORCH_TO_MG[vals.dtype], samples.data_ptr(), samples.shape[0],
                                         out.data_ptr(), _stream(stream)))
        return out


def mg_bitstream_write(g: Graph, stream=None) -> Bitstream:
    """The graph's bitstream (Sec. 3.3, Table 1) encoded on the GPU."""
    n = ctypes.c_size_t()
    _check(lib().mg_bitstream_size(g.handle, ctypes.byref(n)))
    data = torch.empty(n.value, dtype=torch.uint8, device=torch.device("cuda", g.device))
    _check(lib().mg_bitstream_write(g.handle, data.data_ptr(), n.value, _stream(stream)))
    return Bitstream(data)


_STRATEGY = {"occurrence": 1, "reduction": 2}


def mg_factor_greedy(ids: torch.Tensor, num_segments: int, strategy: str = "reduction", tau: int = 3,
                     bitrate: int = 9, graph: bool = False, stream=None) -> dict:
    """Greedy factorisation (phi_1 'occurrence' or phi_2 'reduction') of a
    (nz, ny, nx) uint16/uint32 CUDA volume on the GPU.  Returns a dict with
    the node table (p, q, a, b numpy), the mip IDs of every level, the
    stage-1 picks, the codebook and sigma (bitrate > 0) and the counts."""
    import numpy as np
    if not ids.is_cuda or ids.dim() != 3:
        raise ValueError("ids must be a 3-D CUDA tensor (z, y, x)")
    ids = ids.contiguous()
    nb = 2 if ids.dtype == torch.uint16 else 4
    nz, ny, nx = ids.shape
    o = mg_greedy_opts(_STRATEGY[strategy], tau, bitrate)
    h = ctypes.c_void_p()
    with torch.cuda.device(ids.device):
        _check(lib().mg_factor_greedy(ids.data_ptr(), nx, ny, nz, num_segments, ctypes.byref(mg_build_opts(nb)),
                                      ctypes.byref(o), _stream(stream), ctypes.byref(h)))
    try:
        info = mg_greedy_info()
        _check(lib().mg_greedy_info_get(h, ctypes.byref(info)))
        N, L = info.num_nodes, info.levels
        p = np.zeros(N, np.uint32); q = np.zeros(N, np.uint32)
        a = np.zeros(N, np.uint64); b = np.zeros(N, np.uint64)
        _check(lib().mg_greedy_copy_nodes(h, p.ctypes.data, q.ctypes.data, a.ctypes.data, b.ctypes.data))
        dims, mips = [], []
        d = [nx, ny, nz]
        for l in range(L):
            out = np.zeros((d[2], d[1], d[0]), np.uint32)
            _check(lib().mg_greedy_copy_mip(h, l, out.ctypes.data))
            mips.append(out)
            dims.append(tuple(d))
            d = [(v + 1) // 2 for v in d]
        picks = np.zeros((max(info.picks, 1), 2), np.uint32)
        _check(lib().mg_greedy_copy_picks(h, picks.ctypes.data))
        nbins = (1 << bitrate) if bitrate else 1
        cb = np.zeros(nbins); sg = np.zeros(nbins)
        _check(lib().mg_greedy_copy_codebook(h, cb.ctypes.data, sg.ctypes.data))
        res = dict(N=N, D=info.depth, L=L, p=p, q=q, a=a, b=b, mip=mips, dims=dims,
                   picks=picks[:info.picks], codebook=cb, sigma=sg, waves=info.waves, ms=info.ms)
        if graph:
            # mg_graph_from_greedy: the quantised graph, usable by every fp32 entry point
            dev = ids.device.index if ids.device.index is not None else torch.cuda.current_device()
            alloc = torch_allocator(dev)
            gh = ctypes.c_void_p()
            with torch.cuda.device(dev):
                _check(lib().mg_graph_from_greedy(h, ctypes.byref(alloc), _stream(stream), ctypes.byref(gh)))
            res["graph"] = Graph(gh.value, dev, alloc)
        return res
    finally:
        lib().mg_greedy_free(h)


def mg_error_table(g: Graph, stream=None):
    """mg_error_table_build + mg_error_table_copy: the mixture table with
    its Eq. 17 uncertainties as numpy (off, src, mu, dmu)."""
    import numpy as np
    e = ctypes.c_int64()
    with torch.cuda.device(g.device):
        _check(lib().mg_error_table_build(g.handle, ctypes.byref(e), _stream(stream)))
    off = np.zeros(g.N + 1, np.int64)
    src = np.zeros(max(e.value, 1), np.uint32); mu = np.zeros(max(e.value, 1)); dmu = np.zeros(max(e.value, 1))
    _check(lib().mg_error_table_copy(g.handle, off.ctypes.data, src.ctypes.data, mu.ctypes.data, dmu.ctypes.data))
    return off, src[:e.value], mu[:e.value], dmu[:e.value]


def mg_query_lut(g: Graph, boxes: torch.Tensor, errors: bool = True, stream=None):
    """Box histograms summed from the mixture table and their error bars,
    (Q, S) float64 each (errors=False: error bars None).  Builds the table on
    first use."""
    if not boxes.is_cuda or boxes.dtype != torch.int32 or boxes.dim() != 2 or boxes.shape[1] != 6:
        raise ValueError("boxes must be a CUDA int32 tensor of shape (Q, 6)")
    boxes = boxes.contiguous()
    with torch.cuda.device(g.device):
        _check(lib().mg_error_table_build(g.handle, None, _stream(stream)))
    Q = boxes.shape[0]
    hist = torch.empty((Q, g.S), dtype=torch.float64, device=boxes.device)
    err = torch.empty((Q, g.S), dtype=torch.float64, device=boxes.device) if errors else None
    _check(lib().mg_query_lut(g.handle, boxes.data_ptr(), Q, hist.data_ptr(), err.data_ptr() if errors else None,
                              _stream(stream)))
    return hist, err


def mg_sync_status(g: Graph, stream=None):
    """Synchronise and raise MGError if a kernel recorded an error."""
    _check(lib().mg_sync_status(g.handle, _stream(stream)))


def mg_graph_export(g: Graph, stream=None):
    """The graph as a host image (numpy uint8), for mg_graph_import."""
    import numpy as np
    n = ctypes.c_size_t()
    _check(lib().mg_graph_export_size(g.handle, ctypes.byref(n)))
    img = np.empty(n.value, np.uint8)
    with torch.cuda.device(g.device):
        _check(lib().mg_graph_export(g.handle, img.ctypes.data, img.nbytes, _stream(stream)))
    return img


def mg_graph_import(image, device: int = None, stream=None, use_torch_allocator: bool = True) -> Graph:
    """A graph re-created from an image of mg_graph_export (bytes-like or numpy)."""
    import numpy as np
    img = np.ascontiguousarray(np.frombuffer(image, np.uint8) if not isinstance(image, np.ndarray) else image)
    dev = torch.cuda.current_device() if device is None else device
    alloc = torch_allocator(dev) if use_torch_allocator else None
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        _check(lib().mg_graph_import(img.ctypes.data, img.nbytes, ctypes.byref(alloc) if alloc is not None else None,
                                     _stream(stream), ctypes.byref(h)))
    return Graph(h.value, dev, alloc)


def mg_selftest_bounded_wait(satisfied: bool, spin_limit: int = 1 << 16, stream=None) -> int:
    """Status of a bounded device wait on a flag that is set (MG_OK) or never
    set (MG_ERR_TIMEOUT); raises only for bad arguments or CUDA errors."""
    st = lib().mg_selftest_bounded_wait(1 if satisfied else 0, spin_limit, _stream(stream))
    if st not in (MG_OK, MG_ERR_TIMEOUT):
        _check(st)
    return st


def mg_free(g: Graph):
    lib().mg_free(g.handle)


# --------------------------------------------------------------------------
# request loop (mg_server_*)
# --------------------------------------------------------------------------
_NP_STORAGE = {"f32": "float32", "f16": "float16", "bf16": "uint16"}   # bf16 results as raw bits


class Server:
    """A request loop over resident volumes (mg_server_*).

    Results land in numpy arrays owned by this object until the request is
    waited for; box results are (S,) uint32 (hist='u32') or float32, TF frames
    (P, C) in the storage dtype (bf16 as raw uint16 bits)."""

    def __init__(self, slots: int = 4, max_batch: int = 1024, hist: str = "u32", storage: str = "f32",
                 max_samples: int = 65536, memory_budget: int = 0, plain: bool = False):
        import numpy as np
        self._np = np
        o = mg_server_opts()
        o.slots, o.max_batch = slots, max_batch
        o.hist_type = MG_HIST_F32 if hist == "f32" else MG_HIST_U32
        o.storage = _DTYPES[storage][0]
        o.max_samples, o.memory_budget, o.plain = max_samples, memory_budget, 1 if plain else 0
        h = ctypes.c_void_p()
        _check(lib().mg_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value
        self.hist_dtype = np.float32 if hist == "f32" else np.uint32
        self.storage_dtype = np.dtype(_NP_STORAGE[storage])
        self.volumes = []      # (graph, C)
        self._live = {}        # ticket -> objects the library writes or reads

    def add_volume(self, g: Graph, C: int = 4) -> int:
        v = ctypes.c_int(-1)
        with torch.cuda.device(g.device):
            _check(lib().mg_server_add_volume(self.handle, g.handle, C, ctypes.byref(v)))
        self.volumes.append((g, C))
        return v.value

    def remove_volume(self, volume: int, timeout: float = 0.0):
        """Evict a volume once its queued and running requests are done."""
        _check(lib().mg_server_remove_volume(self.handle, volume, timeout))

    def start(self):
        _check(lib().mg_server_start(self.handle))

    def _request(self, kind, volume, box=None, tf=None, samples=None, out=None, arrival=0.0):
        np = self._np
        r = mg_request()
        r.kind, r.volume, r.arrival_s = kind, volume, float(arrival)
        keep = []
        g, C = self.volumes[volume] if 0 <= volume < len(self.volumes) else (None, 0)
        if kind == MG_REQ_BOX:
            for k in range(6):
                r.box[k] = int(box[k])
            if out is None and g is not None:
                out = np.empty(g.S, self.hist_dtype)
        else:
            tf = np.ascontiguousarray(tf, np.float32)
            keep.append(tf)
            r.tf = tf.ctypes.data
            P = 0
            if samples is not None:
                samples = np.ascontiguousarray(samples, np.float32)
                keep.append(samples)
                r.samples = samples.ctypes.data
                P = samples.shape[0]
            r.P = P
            if out is None:
                out = np.empty((P, C), self.storage_dtype)
        if out is not None:
            r.result = out.ctypes.data
        keep.append(out)
        return r, out, keep

    def submit_box(self, volume: int, box, out=None):
        """Queue a box-histogram request; returns (ticket, result array)."""
        r, out, keep = self._request(MG_REQ_BOX, volume, box=box, out=out)
        t = ctypes.c_uint64()
        _check(lib().mg_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._live[t.value] = keep
        return t.value, out

    def submit_tf(self, volume: int, tf, samples=None, out=None):
        """Queue a TF frame (propagate tf (S, C), look up samples (P, 4)); returns (ticket, result array)."""
        r, out, keep = self._request(MG_REQ_TF, volume, tf=tf, samples=samples, out=out)
        t = ctypes.c_uint64()
        _check(lib().mg_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._live[t.value] = keep
        return t.value, out

    def wait(self, ticket: int, timeout: float = 0.0) -> float:
        """Wait for a request; returns its latency in seconds (raises MGError on failure)."""
        lat = ctypes.c_double()
        st = lib().mg_server_wait(self.handle, ticket, timeout, ctypes.byref(lat))
        if st != MG_ERR_TIMEOUT:
            self._live.pop(ticket, None)
        _check(st)
        return lat.value

    def cancel(self, ticket: int):
        _check(lib().mg_server_cancel(self.handle, ticket))

    def replay(self, requests):
        """Replay a timed stream.  requests: dicts with kind ('box' | 'tf'),
        volume, arrival (s) and box, or tf (+ samples).  Returns
        (results, latencies (n,) seconds, wall seconds)."""
        np = self._np
        n = len(requests)
        arr = (mg_request * max(n, 1))()
        results, keep = [], []
        for i, q in enumerate(requests):
            if q["kind"] == "box":
                r, out, k = self._request(MG_REQ_BOX, q["volume"], box=q["box"], out=q.get("out"),
                                          arrival=q["arrival"])
            else:
                r, out, k = self._request(MG_REQ_TF, q["volume"], tf=q["tf"], samples=q.get("samples"),
                                          out=q.get("out"), arrival=q["arrival"])
            arr[i] = r
            results.append(out)
            keep.append(k)
        lat = np.zeros(max(n, 1), np.float64)
        wall = ctypes.c_double()
        _check(lib().mg_server_replay(self.handle, arr, n, lat.ctypes.data, ctypes.byref(wall)))
        return results, lat[:n], wall.value

    def stats(self) -> dict:
        s = mg_server_stats()
        _check(lib().mg_server_stats_get(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in mg_server_stats._fields_}

    def close(self):
        if self.handle:
            lib().mg_server_free(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_server_create(**kw) -> Server:
    return Server(**kw)
