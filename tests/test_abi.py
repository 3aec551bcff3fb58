"""The C-ABI library builds, loads and exports every symbol include/dfa.h declares (CPU)."""
import ctypes
import os
import re

import pytest

import paper_2508_20735_gb300 as g


@pytest.fixture(scope="module")
def built():
    g.build()
    return g.lib()


def test_header_declares_the_boundary():
    names = set(g.header_functions())
    for must in ["dfa_minimise", "dfa_minimise_batch", "dfa_equivalent", "dfa_workspace_size",
                 "dfa_batch_workspace_size", "dfa_equivalent_workspace_size", "dfa_serve_create",
                 "dfa_serve_submit", "dfa_serve_poll", "dfa_serve_wait", "dfa_serve_stats", "dfa_serve_destroy",
                 "dfa_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(built):
    for name in g.header_functions():
        assert hasattr(built, name), name


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in g._SIGS}
    assert set(g.header_functions()) <= bound


def test_version_and_error_strings(built):
    assert b"sm_103a" in built.dfa_version()
    assert isinstance(built.dfa_last_error(), bytes)


def test_struct_layouts_match_header():
    # dfa_t: two u32, two pointers, u32 (+pad) ; dfa_opts: i32,u32,u64,i32,u32 ; dfa_result: 4 x 32-bit + u64
    assert ctypes.sizeof(g.DfaT) == 32
    assert ctypes.sizeof(g.DfaOpts) == 24
    assert ctypes.sizeof(g.DfaResult) == 24


def test_argument_errors_need_no_gpu(built):
    """Invalid arguments are rejected by host checks before any CUDA call."""
    import numpy as np
    d, keep = g.make_dfa(np.zeros((1, 4), np.uint32), np.zeros(4, np.uint8), start=0)
    d.n = 0
    assert g.dfa_workspace_size(d, None) == 0
    st, _ = g.dfa_minimise(d, None, 1, 256, 1 << 20, None)
    assert st == g.DFA_EINVAL and "n = 0" in g.last_error()
    d.n = 4
    d.start = 9
    st, _ = g.dfa_minimise(d, None, 1, 256, 1 << 20, None)
    assert st == g.DFA_EINVAL and "start" in g.last_error()
    a, ka = g.make_dfa(np.zeros((1, 4), np.uint32), np.zeros(4, np.uint8))
    b, kb = g.make_dfa(np.zeros((2, 4), np.uint32), np.zeros(4, np.uint8))
    st, eq, _ = g.dfa_equivalent(a, b, None, 256, 1 << 20, None)
    assert st == g.DFA_EINVAL and "alphabets differ" in g.last_error()


def test_noalloc_argument_errors_need_no_gpu(built):
    """dfa_minimise_noalloc rejects, before any launch, an algorithm other than
    signature refinement and host (numpy) arrays."""
    import numpy as np
    delta = np.zeros((2, 8), np.uint32)
    acc = np.zeros(8, np.uint8)
    out = np.zeros(8, np.uint32)
    d, keep = g.make_dfa(delta, acc)
    st, _ = g.dfa_minimise_noalloc(d, g.make_opts("closure_moore"), out.ctypes.data, None)
    assert st == g.DFA_EINVAL and "signature refinement only" in g.last_error()
    st, _ = g.dfa_minimise_noalloc(d, None, out.ctypes.data, None)
    assert st == g.DFA_EINVAL and "device pointers" in g.last_error()


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle and has no numpy refinement code."""
    pkg = os.path.dirname(g.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
