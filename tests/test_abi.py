"""The C-ABI library builds, loads without a GPU, and exports every symbol gr.h declares.

No compute call is made here (this runs on machines without a GPU).
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1701_01170_gb300 import _build
    try:
        _build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gr_graph_create_csr", "gr_advance", "gr_filter", "gr_bfs", "gr_sssp",
                     "gr_sync_status", "gr_graph_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in gr.h but not exported: {missing}"


def test_exports_are_c_linkage(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (gr_[a-z0-9_]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_status_strings_without_gpu(lib_path):
    import paper_1701_01170_gb300 as gr
    gr.load()
    assert gr.status_str(gr.GR_OK) == "GR_OK"
    assert gr.status_str(gr.GR_ERR_TIMEOUT) == "GR_ERR_TIMEOUT"
    assert gr.status_str(-99) == "GR_ERR_UNKNOWN"
    assert gr.gr_version() >> 16 == 1


def test_option_struct_layouts_match_header(lib_path):
    import paper_1701_01170_gb300 as gr
    o = gr.bfs_opts()
    assert o.direction == gr.GR_DIR_AUTO and o.big_degree > 0 and o.spin_limit > 0
    s = gr.sssp_opts()
    assert s.delta == 0 and s.big_degree > 0
    assert ctypes.sizeof(gr.gr_bfs_opts) == 56
    assert ctypes.sizeof(gr.gr_sssp_opts) == 48
    assert ctypes.sizeof(gr.gr_bfs_state) == 24
    assert ctypes.sizeof(gr.gr_sssp_state) == 16


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1701_01170_gb300 as gr
    from paper_1701_01170_gb300 import _build
    monkeypatch.setattr(gr, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        gr.load()


def test_ctypes_mirrors_match_the_compiled_header(tmp_path):
    # compile gr.h with the host C compiler and compare every struct's size
    # and field offsets with the ctypes mirror of the Python binding
    import shutil

    import paper_1701_01170_gb300 as gr
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [gr.gr_run_stats, gr.gr_bfs_state, gr.gr_sssp_state, gr.gr_bfs_opts,
               gr.gr_sssp_opts, gr.gr_msbfs_opts, gr.gr_job, gr.gr_batch_opts]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gr.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in st._fields_:
            lines.append(f'  printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st in structs:
        name = st.__name__
        assert int(got[name]) == ctypes.sizeof(st), name
        for f in st._fields_:
            assert int(got[f"{name}.{f[0]}"]) == getattr(st, f[0]).offset, (name, f[0])


def test_binding_rejects_narrow_or_short_output_tensors():
    # the kernels write n 32-bit values through each output pointer: the
    # binding refuses tensors that would be overrun, before any GPU call
    import torch

    import paper_1701_01170_gb300 as gr
    with pytest.raises(ValueError, match="32-bit"):
        gr._buf32(torch.zeros(10, dtype=torch.int16), 10, "depth")
    with pytest.raises(ValueError, match="32-bit"):
        gr._buf32(torch.zeros(10, dtype=torch.int64), 10, "depth")
    with pytest.raises(ValueError, match="needs 10 elements"):
        gr._buf32(torch.zeros(9, dtype=torch.int32), 10, "dist")
    with pytest.raises(ValueError, match="CUDA"):        # right size, but host memory
        gr._buf32(torch.zeros(10, dtype=torch.int32), 10, "pred")
    assert gr._buf32(None, 10, "pred") is None           # optional outputs stay optional


def test_option_builders_reject_unknown_fields(lib_path):
    import paper_1701_01170_gb300 as gr
    for build in (gr.bfs_opts, gr.sssp_opts, gr.msbfs_opts, gr.batch_opts):
        with pytest.raises(TypeError, match="no field"):
            build(no_such_field=1)
    assert gr.msbfs_opts(snapshot_levels=3).snapshot_levels == 3
    assert gr.batch_opts(cluster_size=4).cluster_size == 4


def test_load_refuses_a_library_missing_declared_symbols(tmp_path, monkeypatch):
    # an out-of-date or foreign libgr.so must not load with some entry points unbound
    import shutil

    import paper_1701_01170_gb300 as gr
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "stub.c"
    src.write_text("int gr_version(void) { return 1 << 16; }\n")
    so = tmp_path / "libstub.so"
    subprocess.check_call([cc, "-shared", "-fPIC", str(src), "-o", str(so)])
    monkeypatch.setattr(gr, "_lib", None)
    monkeypatch.setenv("GR_LIBRARY", str(so))
    with pytest.raises(RuntimeError, match="does not export"):
        gr.load()
