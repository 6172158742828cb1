"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/mg.h declares, and rejects bad arguments on the host
before any launch."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


def _declared():
    with open(os.path.join(ROOT, "include", "mg.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"MG_API\s+[\w\s\*]+?\b(mg_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_02702_gb300 import build as b
    b.build_mg()
    from paper_2009_02702_gb300 import mg
    return mg.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mg_build", "mg_propagate_tf", "mg_query_boxes", "mg_render_lookup", "mg_free", "mg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2009_02702_gb300 import mg
    names = _declared()
    assert sorted(mg.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_host_argument_checks(lib):
    from paper_2009_02702_gb300 import mg
    h = ctypes.c_void_p()
    opts = mg.mg_build_opts(2)
    # NULL ids, bad dims, bad id width: rejected before touching the device
    assert lib.mg_build(None, 4, 4, 4, 3, ctypes.byref(opts), None, None, ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG
    assert "ids" in mg.mg_last_error()
    assert lib.mg_build(ctypes.c_void_p(16), 0, 4, 4, 3, ctypes.byref(opts), None, None,
                        ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_build(ctypes.c_void_p(16), 70000, 4, 4, 3, ctypes.byref(opts), None, None,
                        ctypes.byref(h)) == mg.MG_ERR_UNSUPPORTED
    bad = mg.mg_build_opts(3)
    assert lib.mg_build(ctypes.c_void_p(16), 4, 4, 4, 3, ctypes.byref(bad), None, None,
                        ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_build(ctypes.c_void_p(16), 4, 4, 4, 0, ctypes.byref(opts), None, None,
                        ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG
    # NULL graph
    o = mg.mg_query_opts()
    assert lib.mg_query_boxes(None, None, 0, ctypes.byref(o), None, 0, None, None, None, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_propagate_tf(None, None, 4, 0, None, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_render_lookup(None, None, 4, 0, None, 0, None, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_count_cubes(None, None, 0, None, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_sync_status(None, None) == mg.MG_ERR_INVALID_ARG
    f = ctypes.c_float()
    assert lib.mg_query_plan_timing(None, ctypes.byref(f), ctypes.byref(f)) == mg.MG_ERR_INVALID_ARG
    lib.mg_free(None)
    assert mg.mg_version().startswith("mixgraph-gb300")


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2009_02702_gb300 import mg
    monkeypatch.setattr(mg, "_lib", None)
    monkeypatch.setattr(mg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        mg.lib()


def test_server_host_argument_checks(lib):
    """Request-loop options and handles are checked before any CUDA call."""
    from paper_2009_02702_gb300 import mg
    h = ctypes.c_void_p()
    assert lib.mg_server_create(None, None) == mg.MG_ERR_INVALID_ARG
    for field, value in (("slots", 65), ("slots", -1), ("max_batch", -3), ("max_batch", (1 << 20) + 1),
                         ("hist_type", 2), ("storage", 7), ("memory_budget", -1), ("plain", 2),
                         ("max_samples", -5)):
        o = mg.mg_server_opts()
        setattr(o, field, value)
        assert lib.mg_server_create(ctypes.byref(o), ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG, field
        assert h.value is None
    v = ctypes.c_int()
    assert lib.mg_server_add_volume(None, None, 4, ctypes.byref(v)) == mg.MG_ERR_INVALID_ARG
    r = mg.mg_request()
    t = ctypes.c_uint64()
    assert lib.mg_server_submit(None, ctypes.byref(r), ctypes.byref(t)) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_server_start(None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_server_cancel(None, 0) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_server_wait(None, 0, 0.0, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_server_replay(None, None, 0, None, None) == mg.MG_ERR_INVALID_ARG
    s = mg.mg_server_stats()
    assert lib.mg_server_stats_get(None, ctypes.byref(s)) == mg.MG_ERR_INVALID_ARG
    lib.mg_server_free(None)


def test_server_struct_layout_matches_header():
    """The binding's ctypes structs have the sizes the C compiler gives the header's."""
    import shutil
    import subprocess
    from paper_2009_02702_gb300 import mg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    work = os.path.join(ROOT, "tests", "_build")
    os.makedirs(work, exist_ok=True)
    src = os.path.join(work, "layout.c")
    exe = os.path.join(work, "layout")
    with open(src, "w") as f:
        f.write('#include <stdio.h>\n#include "mg.h"\nint main(void){printf("%zu %zu %zu %zu %zu",'
                "sizeof(mg_server_opts),sizeof(mg_request),sizeof(mg_server_stats),sizeof(mg_query_opts),"
                "sizeof(mg_graph_info));printf(\" %zu\",sizeof(mg_camera));return 0;}\n")
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), src, "-o", exe])
    sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(mg.mg_server_opts), ctypes.sizeof(mg.mg_request),
                     ctypes.sizeof(mg.mg_server_stats), ctypes.sizeof(mg.mg_query_opts),
                     ctypes.sizeof(mg.mg_graph_info), ctypes.sizeof(mg.mg_camera)]


def test_selftest_wait_argument_checks(lib):
    from paper_2009_02702_gb300 import mg
    assert lib.mg_selftest_bounded_wait(2, 10, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_selftest_bounded_wait(0, 0, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_selftest_bounded_wait(0, (1 << 22) + 1, None) == mg.MG_ERR_INVALID_ARG


def test_graph_io_argument_checks(lib):
    from paper_2009_02702_gb300 import mg
    n = ctypes.c_size_t()
    h = ctypes.c_void_p()
    assert lib.mg_graph_export_size(None, ctypes.byref(n)) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_graph_export(None, None, 0, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_graph_import(None, 0, None, None, ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG
    junk = (ctypes.c_uint8 * 4096)()
    assert lib.mg_graph_import(junk, 4096, None, None, ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_graph_import(junk, 10, None, None, ctypes.byref(h)) == mg.MG_ERR_INVALID_ARG


def test_output_tensor_checks():
    # caller outputs are written through their data pointers: contiguous, and
    # the result's shape, dtype and device, else ValueError before any call
    torch = pytest.importorskip("torch")
    from paper_2009_02702_gb300 import mg
    cpu = torch.device("cpu")
    ok = torch.empty((5, 7), dtype=torch.uint32)
    assert mg._check_out(ok, (5, 7), torch.uint32, cpu) is ok
    bad = [torch.empty((5, 7), dtype=torch.float32), torch.empty((7, 5), dtype=torch.uint32),
           torch.empty((5, 14), dtype=torch.uint32)[:, ::2], torch.empty(35, dtype=torch.uint32), None]
    for b in bad:
        with pytest.raises(ValueError):
            mg._check_out(b, (5, 7), torch.uint32, cpu)
    with pytest.raises(ValueError):
        mg._check_out(ok, (5, 7), torch.uint32, torch.device("cuda", 0))


def test_noalloc_binding_checks_the_output(monkeypatch):
    # the fixed-scratch query writes Q*S uint32 through out's data pointer: an
    # output of another dtype, shape or layout is refused before the library
    # is called (here a stand-in that fails the test if it is reached)
    torch = pytest.importorskip("torch")
    from types import SimpleNamespace
    from paper_2009_02702_gb300 import mg

    def unreachable():
        raise AssertionError("the library was called with a bad output")
    monkeypatch.setattr(mg, "lib", unreachable)
    boxes = SimpleNamespace(is_cuda=True, dtype=torch.int32, shape=(5, 6), device=torch.device("cpu"),
                            dim=lambda: 2)
    boxes.contiguous = lambda: boxes
    g = SimpleNamespace(S=7, handle=None)
    bad = [torch.empty((5, 7), dtype=torch.uint8), torch.empty((5, 7), dtype=torch.int16),
           torch.empty((5, 7), dtype=torch.float32), torch.empty((7, 5), dtype=torch.uint32),
           torch.empty((5, 14), dtype=torch.uint32)[:, ::2], torch.empty(35, dtype=torch.uint32)]
    for b in bad:
        with pytest.raises(ValueError):
            mg.mg_query_boxes_noalloc(g, boxes, out=b)
