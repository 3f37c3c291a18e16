"""CPU-side checks of the CUDA library: it loads without a GPU and exports
every function that include/mce.h declares; host-side logic only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?!typedef)(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("mce_graph_create", "mce_enumerate", "mce_rank", "imce_open", "imce_add_edges",
                 "mce_enumerate_batched", "mce_model_train"):
        assert must in names


def test_library_loads_and_exports_every_symbol():
    import paper_2001_11433_gb300 as mce
    lib = mce.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(mce.SIGNATURES)


def test_host_only_calls():
    import paper_2001_11433_gb300 as mce
    lib = mce.load()
    assert lib.mce_strerror(mce.MCE_EOVERFLOW).startswith(b"output buffer")
    o = mce.Opts()
    lib.mce_opts_init(ctypes.byref(o))
    assert o.rank_kind == mce.RANK_DEGEN and o.split == 1 and o.node_budget == 0
    assert lib.mce_kernel_launches() == 0
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert lib.mce_graph_create(None, None, -1, 10, 1, None, ctypes.byref(h)) == mce.MCE_EINVAL
    assert lib.mce_enumerate(None, None, None) == mce.MCE_EINVAL


def test_kernel_sources_target_sm103a_only():
    from paper_2001_11433_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
